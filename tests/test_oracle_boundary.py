"""Pins of the oracle's boundary rule (Sec. 3.1.1, Alg. 1, Remark 1) and 2^n
subdivision (Sec. 2.1): the worked example of Fig. 4, brute force over every
leaf, and the union-preserving split."""
import os

import numpy as np
import pytest

from paper_2202_06111_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


def _identity(n, n0, lo=0.0, hi=None):
    hi = float(n0) if hi is None else hi
    dyn = W.linmap(np.eye(n).tolist(), np.zeros((n, 1)).tolist())
    return W.problem(dyn, [lo] * n, [hi] * n, n0, 2, [[0.0]], 1.0, 0)


def test_fig4_boundary_selection(orc):
    """B_1..B_25 on a 5 x 5 covering, numbered row by row (tests/golden/fig4_boundary.txt)."""
    rows = [ln.split() for ln in open(os.path.join(HERE, "golden", "fig4_boundary.txt"))
            if ln.strip() and not ln.startswith("#")]
    for case, removed, cell, want in rows:
        s = orc.Solver(_identity(2, 5))
        s.build_graph()
        lv, idx = s.live()
        slot = {tuple(r): i for i, r in enumerate(idx)}

        def B(i):
            r, c = divmod(i - 1, 5)
            return slot[(c, r)]
        kept = np.ones(len(lv), np.uint8)
        for b in removed.split(","):
            kept[B(int(b))] = 0
        s.set_kept(kept)
        bnd = s.classify()
        assert bnd[B(int(cell))] == bool(int(want)), (case, cell)


def _bruteforce_boundary(prob, s, bnd):
    """Exact: a kept leaf is boundary iff it touches a face of X or any removed
    leaf's closed box meets its closed box (integer coordinates on the finest grid)."""
    n = prob["n"]
    lv, st, idx, ch = s.nodes()
    F = s.max_level()
    leaf = st != 2
    scale = (1 << (F - lv))[:, None]
    a, b = idx * scale, (idx + 1) * scale
    N = np.array(prob["n0"][:n]) << F
    live_lv, live_idx = s.live()
    kept = s.kept()
    for i, (L, r) in enumerate(zip(live_lv, live_idx)):
        if not kept[i]:
            assert not bnd[i]
            continue
        f = 1 << (F - L)
        ca, cb = np.array(r) * f, (np.array(r) + 1) * f
        face = bool(np.any(ca == 0) or np.any(cb == N))
        meet = np.all((a <= cb[None, :]) & (b >= ca[None, :]), axis=1)
        dead = bool(np.any(meet & leaf & (st == 0)))
        assert bool(bnd[i]) == (face or dead), (L, r)


@pytest.mark.parametrize("rule", ["outer", "inner"])
def test_boundary_bruteforce_multilevel(orc, rule):
    prob = W.problem(W.vdp(1.0), [-4, -4], [4, 4], 8, 3, W.controls_grid(-1, 1, 3), 0.25, 2, rule=rule)
    s = orc.Solver(prob)
    for L in range(4):
        s.build_graph()
        s.prune()
        bnd = s.classify()
        _bruteforce_boundary(prob, s, bnd)
        if L < 3:
            s.subdivide()


def test_subdivision_children_and_union(orc):
    """Boundary cells split into 2^n children 2 idx + bits at level + 1; the
    leaves (kept, removed and new) still tile X exactly."""
    prob = W.problem(W.vdp(1.0), [-4, -4], [4, 4], 8, 3, W.controls_grid(-1, 1, 3), 0.25, 2, rule="outer")
    s = orc.Solver(prob)
    for L in range(3):
        s.build_graph()
        s.prune()
        before = {(int(a),) + tuple(map(int, b)) for a, b in zip(*s.live())}
        bnd = s.classify()
        lv_live, idx_live = s.live()
        split = {(int(a),) + tuple(map(int, b)) for a, b, f in zip(lv_live, idx_live, bnd) if f}
        ns = s.subdivide()
        assert ns == len(split)
        s.build_graph()
        after = {(int(a),) + tuple(map(int, b)) for a, b in zip(*s.live())}
        kids = {(L0 + 1, 2 * i + bi, 2 * j + bj) for (L0, i, j) in split for bi in (0, 1) for bj in (0, 1)}
        assert kids <= after
        assert after - kids <= before
        lv, st, idx, ch = s.nodes()
        F = s.max_level()
        area = sum(4 ** (F - int(l)) for l, t in zip(lv, st) if t != 2)
        assert area == (8 << F) ** 2


def _touch(a_lo, a_hi, b_lo, b_hi):
    """Closed boxes (per-dimension integer bounds at the finest level) meet."""
    return bool(np.all(a_lo <= b_hi) and np.all(b_lo <= a_hi))


@pytest.mark.parametrize("ring", [1, 2, -1])
def test_split_rings_brute_force(orc, ring):
    """The rings that stand in for the N nearest neighbours (Sec. 3.1.2): ring r
    adds the kept cells whose closed boxes meet a cell of ring r - 1, ring 0
    being the exact boundary cells; -1 splits every kept cell. Checked at a
    refined level (leaves of two levels) against brute force over closed boxes
    in integer coordinates of the finest level."""
    base = W.problem(W.vdp(1.0), [-3, -3], [3, 3], 8, 3, W.controls_grid(-1, 1, 3), 0.25, 2, rule="outer",
                     precision="fp64")
    s = orc.Solver(dict(base, split_ring=ring))
    s.build_graph()
    s.prune()
    s.subdivide()
    s.build_graph()
    s.prune()
    lv, idx = s.live()
    kept = s.kept()
    F = int(lv.max())
    lo = idx.astype(np.int64) << (F - lv[:, None])
    hi = (idx.astype(np.int64) + 1) << (F - lv[:, None])
    top = np.array(base["n0"], np.int64) << F
    # removed leaves: the removed cells of this level and the removed leaves of the tree
    nl, nst, nidx, _ = s.nodes()
    dead = [(nidx[j].astype(np.int64) << (F - nl[j]), (nidx[j].astype(np.int64) + 1) << (F - nl[j]))
            for j in range(len(nl)) if nst[j] == orc.DEAD]
    dead += [(lo[c], hi[c]) for c in range(len(lv)) if not kept[c]]
    mark = np.zeros(len(lv), bool)
    for c in range(len(lv)):
        if kept[c]:
            mark[c] = bool(np.any(lo[c] == 0) or np.any(hi[c] == top)) or \
                any(_touch(lo[c], hi[c], a, b) for a, b in dead)
    want0 = mark.copy()
    if ring == -1:
        mark = kept.copy()
    for _ in range(max(ring, 0)):
        nxt = mark.copy()
        for c in range(len(lv)):
            if kept[c] and not mark[c]:
                nxt[c] = any(mark[o] and _touch(lo[c], hi[c], lo[o], hi[o]) for o in range(len(lv)))
        mark = nxt
    got = s.classify()
    # (all-split leaves one live level; the removed root cells stay as leaves)
    assert len(set(lv.tolist())) == (1 if ring == -1 else 2)
    assert 0 < want0.sum() < mark.sum() <= kept.sum()
    assert np.array_equal(got, mark)


@pytest.mark.parametrize("ring", [0, 1])
def test_boundary_cycled_bisection_brute_force(orc, ring):
    """With cycled bisection (2 children, halving dimension depth mod n) the
    boundary rule and its rings use the same closed-touch relation: brute force
    in integer coordinates of the finest halvings of each dimension."""
    base = dict(W.problem(W.vdp(1.0), [-3, -3], [3, 3], 8, 3, W.controls_grid(-1, 1, 3), 0.25, 2, rule="outer",
                          precision="fp64"), split="cycled", split_ring=ring)
    s = orc.Solver(base)
    for _ in range(3):
        s.build_graph()
        s.prune()
        s.subdivide()
    s.build_graph()
    s.prune()
    lv, idx = s.live()
    kept = s.kept()
    n = 2

    def dlev(L):
        return np.array([L // n + (d < L % n) for d in range(n)], np.int64)
    nl, nst, nidx, _ = s.nodes()
    F = np.max([dlev(int(L)) for L in nl], axis=0)
    top = np.array(base["n0"], np.int64) << F

    def box(L, i):
        sh = F - dlev(int(L))
        return np.asarray(i, np.int64) << sh, (np.asarray(i, np.int64) + 1) << sh
    lo_hi = [box(lv[c], idx[c]) for c in range(len(lv))]
    dead = [box(nl[j], nidx[j]) for j in range(len(nl)) if nst[j] == orc.DEAD]
    dead += [lo_hi[c] for c in range(len(lv)) if not kept[c]]
    mark = np.zeros(len(lv), bool)
    for c in range(len(lv)):
        if kept[c]:
            a, b = lo_hi[c]
            mark[c] = bool(np.any(a == 0) or np.any(b == top)) or any(_touch(a, b, x, y) for x, y in dead)
    for _ in range(ring):
        nxt = mark.copy()
        for c in range(len(lv)):
            if kept[c] and not mark[c]:
                nxt[c] = any(mark[o] and _touch(*lo_hi[c], *lo_hi[o]) for o in range(len(lv)))
        mark = nxt
    got = s.classify()
    assert len(set(lv.tolist())) >= 2 and 0 < mark.sum() <= kept.sum()
    assert np.array_equal(got, mark)
