"""Pins of the oracle's sample lattice, image box and symbolic-image edges
(Def. 1 with closed cells, Sec. 2.1 coverings) against exact geometry and
brute force over every leaf of the subdivision tree."""
import itertools

import numpy as np
import pytest

from paper_2202_06111_gb300 import workloads as W


def _identity(n, n0, lo=-4.0, hi=4.0, k=2):
    dyn = W.linmap(np.eye(n).tolist(), np.zeros((n, 1)).tolist())
    return W.problem(dyn, [lo] * n, [hi] * n, n0, k, [[0.0]], 1.0, 0)


def test_sample_lattice(orc):
    """k = 2 gives exactly the 2^n corners; k = 3 adds the mid-points (dyadic grid)."""
    p = _identity(2, 8)
    s = orc.cell_samples(p, 0, [3, 5])
    assert sorted(map(tuple, s)) == [(-1.0, 1.0), (-1.0, 2.0), (0.0, 1.0), (0.0, 2.0)]
    p3 = dict(_identity(2, 8, k=3))
    s = orc.cell_samples(p3, 1, [6, 9])       # level 1: width 0.5, box [-1,-0.5] x [0.5,1]
    xs = sorted(set(s[:, 0]))
    ys = sorted(set(s[:, 1]))
    assert xs == [-1.0, -0.75, -0.5] and ys == [0.5, 0.75, 1.0] and len(s) == 9
    p1 = dict(_identity(2, 8, k=1))
    assert list(orc.cell_samples(p1, 0, [0, 0])[0]) == [-3.5, -3.5]


def test_level_range_closed_touch(orc):
    """A box edge on a grid line meets the cells on both sides (closed cells);
    ranges are cut to the cells of X and empty outside it."""
    p = _identity(1, 8)                       # X = [-4, 4], w = 1
    assert orc.level_range(p, 0, 0, 0.0, 0.0) == (3, 4)      # the line between cells 3 and 4
    assert orc.level_range(p, 0, 0, 0.25, 0.75) == (4, 4)
    assert orc.level_range(p, 0, 0, -0.5, 1.0) == (3, 5)
    assert orc.level_range(p, 0, 0, -10.0, -4.0) == (0, 0)   # touches the face of X
    lo, hi = orc.level_range(p, 0, 0, -10.0, -4.5)           # outside: empty
    assert lo > hi
    assert orc.level_range(p, 0, 0, 3.5, 9.0) == (7, 7)
    assert orc.level_range(p, 2, 0, 0.0, 0.0) == (15, 16)    # level 2, w = 1/4


@pytest.mark.parametrize("n,n0", [(1, 8), (2, 8), (3, 4)])
def test_identity_map_gives_closed_neighbourhood(orc, n, n0):
    """Identity map with corner samples: the image box is the cell itself, so
    its targets are the 3^n closed neighbourhood (cut at the faces of X)."""
    s = orc.Solver(_identity(n, n0))
    s.build_graph()
    lv, idx = s.live()
    off, tgt, flag, _ = s.graph()
    assert np.all(flag == orc.F_INX)
    key = {tuple(r): i for i, r in enumerate(idx)}
    for i, r in enumerate(idx):
        want = sorted(key[c] for c in itertools.product(*[range(max(0, v - 1), min(n0, v + 2)) for v in r]))
        assert list(tgt[off[i]:off[i + 1]]) == want


def _dlev(prob, lv):
    """Halvings per dimension of cells at depths lv: the depth itself, or with
    cycled bisection depth // n plus one for the dimensions below depth % n."""
    n = prob["n"]
    lv = np.asarray(lv)[:, None]
    if prob.get("split", "all") != "cycled":
        return np.repeat(lv, n, axis=1)
    d = np.arange(n)[None, :]
    return lv // n + (d < lv % n)


def _tree_leaves(s):
    lv, st, idx, ch = s.nodes()
    leaf = st != 2
    return lv[leaf], st[leaf], idx[leaf]


def _bruteforce_graph(prob, s, slack=1e-12):
    """Every leaf (alive or removed) of the tree tested against every image box
    by closed-box overlap. A leaf whose overlap is decided by less than `slack`
    (relative to the box of X) is a rounding tie: the oracle may count it
    either way (its t = (y - lo)/w rounds there), every other leaf must agree."""
    n = prob["n"]
    lo, hi, n0 = np.array(prob["lo"]), np.array(prob["hi"]), np.array(prob["n0"])
    eps = slack * (hi - lo).max()
    llv, lst, lidx = _tree_leaves(s)
    w = (hi - lo)[None, :] / (n0[None, :] * (2.0 ** _dlev(prob, llv)))
    cell_lo = lo[None, :] + lidx * w
    cell_hi = lo[None, :] + (lidx + 1) * w
    live_lv, live_idx = s.live()
    slot = {(int(a),) + tuple(b): i for i, (a, b) in enumerate(zip(live_lv, live_idx))}
    off, tgt, flag, bbox = s.graph()
    ties = 0
    for p in range(len(flag)):
        ymin, ymax = bbox[p, :n], bbox[p, n:]
        g1 = ymax[None, :] - cell_lo          # meet needs g1 >= 0 and g2 >= 0
        g2 = cell_hi - ymin[None, :]
        tie = ((g1 != 0) & (np.abs(g1) < eps)) | ((g2 != 0) & (np.abs(g2) < eps))
        meet = np.all((g1 >= 0) & (g2 >= 0), axis=1)
        sure = meet & ~np.any(tie, axis=1)
        maybe = np.all((g1 > -eps) & (g2 > -eps), axis=1)
        got = set(tgt[off[p]:off[p + 1]].tolist())
        want = {slot[(int(llv[j]),) + tuple(lidx[j])] for j in np.nonzero(sure & (lst == 1))[0]}
        allow = {slot[(int(llv[j]),) + tuple(lidx[j])] for j in np.nonzero(maybe & (lst == 1))[0]}
        assert want <= got <= allow, p
        assert list(tgt[off[p]:off[p + 1]]) == sorted(got)
        dead_sure = bool(np.any(sure & (lst == 0)))
        dead_maybe = bool(np.any(maybe & (lst == 0)))
        f_dead = bool(flag[p] & 2)
        assert dead_sure <= f_dead <= dead_maybe, p
        ties += (want != allow) or (dead_sure != dead_maybe)
        inx = bool(np.all(ymin >= lo) and np.all(ymax <= hi))
        assert bool(flag[p] & 1) == inx, p
    assert ties <= max(2, len(flag) // 20)


@pytest.mark.parametrize("rule", ["outer", "inner"])
def test_targets_bruteforce_multilevel(orc, rule):
    """Van der Pol on a dyadic box, three levels of boundary refinement (removed
    cells at every level): the tree descent finds exactly the leaves the brute
    force finds, and the touches-removed and inside-X flags agree."""
    prob = W.problem(W.vdp(1.0), [-4, -4], [4, 4], 8, 3, W.controls_grid(-1, 1, 3), 0.25, 2,
                     rule=rule)
    s = orc.Solver(prob)
    for L in range(4):
        s.build_graph()
        _bruteforce_graph(prob, s)
        s.prune()
        if L < 3:
            s.subdivide()
    if rule == "outer":
        assert s.max_level() == 3


def test_targets_bruteforce_4d(orc):
    """A 4-D linear map with one refinement level: descent vs brute force."""
    A = [[0.9137, 0.2213, 0.0, 0.0], [-0.3071, 1.1093, 0.1179, 0.0],
         [0.0, 0.0531, 0.8123, 0.3037], [0.1011, 0.0, -0.2093, 1.0517]]
    B = [[0.0], [0.5113], [0.0], [1.0071]]
    prob = W.problem(W.linmap(A, B), [-2] * 4, [2] * 4, 4, 2, W.controls_grid(-0.37, 0.41, 3), 1.0, 0,
                     rule="outer")
    s = orc.Solver(prob)
    s.build_graph()
    _bruteforce_graph(prob, s)
    s.prune()
    s.subdivide()
    s.build_graph()
    _bruteforce_graph(prob, s)


def test_bbox_is_minmax_of_propagated_samples(orc):
    """The stored image box is the per-dimension min / max of f over the samples."""
    prob = W.cstr_256(levels=0, n0=16)
    s = orc.Solver(prob)
    s.build_graph()
    lv, idx = s.live()
    _, _, _, bbox = s.graph()
    ctrl = np.asarray(prob["controls"])
    for slot in (0, 17, 100, 255):
        for u in (0, 5, 10):
            ys = np.array([orc.step(prob, x, ctrl[u]) for x in orc.cell_samples(prob, int(lv[slot]), idx[slot])])
            got = bbox[slot * len(ctrl) + u]
            assert list(got[:2]) == list(ys.min(0)) and list(got[2:]) == list(ys.max(0))


@pytest.mark.parametrize("rule", ["outer", "inner"])
def test_targets_bruteforce_cycled_bisection(orc, rule):
    """Cycled bisection (a split halves dimension depth mod n only): after four
    refinements the covering mixes cells of several shapes; the descent finds
    exactly the leaves the brute force finds."""
    prob = dict(W.problem(W.vdp(1.0), [-4, -4], [4, 4], 8, 3, W.controls_grid(-1, 1, 3), 0.25, 2, rule=rule),
                split="cycled")
    s = orc.Solver(prob)
    for L in range(5):
        s.build_graph()
        _bruteforce_graph(prob, s)
        s.prune()
        if L < 4:
            s.subdivide()
    if rule == "outer":
        assert s.max_level() == 4


def test_cycled_bisection_tiles_X(orc):
    """The leaves (alive and removed) of a cycled-bisection tree tile X: in integer
    coordinates of the finest halvings their boxes fill the grid exactly once."""
    prob = dict(W.problem(W.vdp(1.0), [-4, -4], [4, 4], 6, 3, W.controls_grid(-1, 1, 3), 0.25, 2, rule="outer"),
                split="cycled")
    s = orc.Solver(prob)
    for _ in range(4):
        s.build_graph()
        s.prune()
        s.subdivide()
    lv, st, idx = _tree_leaves(s)
    dl = _dlev(prob, lv)
    F = dl.max(axis=0)
    cover = np.zeros([6 << int(F[0]), 6 << int(F[1])], np.int32)
    for j in range(len(lv)):
        sh = F - dl[j]
        a, b = idx[j] << sh, (idx[j] + 1) << sh
        cover[a[0]:b[0], a[1]:b[1]] += 1
    assert len(set(lv.tolist())) > 2 and np.all(cover == 1)


def test_cycled_bisection_in_one_dimension_is_the_plain_split(orc):
    prob = W.problem(W.linmap([[1.7]], [[1.0]]), [-1.0], [1.0], 12, 3, W.controls_grid(-0.3, 0.3, 3), 1.0, 0,
                     rule="outer")
    res = []
    for split in ("all", "cycled"):
        s = orc.Solver(dict(prob, split=split))
        out = []
        for L in range(4):
            s.build_graph()
            off, tgt, flag, _ = s.graph()
            out.append((s.prune(), off.tolist(), tgt.tolist(), flag.tolist()))
            if L < 3:
                out.append(s.subdivide())
        res.append(out)
    assert res[0] == res[1]



def _overflow_map(rule):
    """x+ = 1e308 x on X = [-4, 4], four cells, corner samples: the corner at
    x = 0 maps to 0, every other corner overflows to +-inf. The cells [-2, 0]
    and [0, 2] therefore have one finite image, 0, inside X."""
    dyn = W.linmap([[1e308]], [[0.0]])
    return dict(W.problem(dyn, [-4.0], [4.0], 4, 2, [[0.0]], 1.0, 0), rule=rule)


@pytest.mark.parametrize("rule", ["inner", "outer"])
def test_nonfinite_image_leaves_x(orc, rule):
    """Reading 8 (the paper defines no image for a sample whose image is not a
    number): a pair with a non-finite sample image leaves X and has no target,
    even where its finite samples land inside X. Mistakes this catches: a box
    and targets taken from the finite samples only (cells [-2, 0] and [0, 2]
    would meet the cells around 0 and stay in X), an infinite extreme let
    through the in-X test, a removed-leaf flag set on such a pair."""
    s = orc.Solver(_overflow_map(rule))
    s.build_graph()
    off, tgt, flag, _ = s.graph()
    assert len(flag) == 4
    assert np.all(flag == orc.F_NONFINITE)
    assert np.all(np.diff(off) == 0) and len(tgt) == 0
    # the finite sample of the two middle cells is still the image of x = 0
    lo, hi, nf = orc.pair_bbox(_overflow_map(rule), 0, [1], [0.0])
    assert nf and lo[0] == 0.0 and hi[0] == 0.0
    assert s.prune() == 0
    assert not s.kept().any()


def test_nonfinite_control_drops_only_its_pairs(orc):
    """Two controls on a contraction: u = 0 keeps x+ = x / 2 inside X, u = 2
    overflows (1e308 * 2 = inf). Only the u = 2 pairs are non-finite and
    target-free, and both rules keep every cell through u = 0."""
    dyn = W.linmap([[0.5]], [[1e308]])
    for rule in ("inner", "outer"):
        p = dict(W.problem(dyn, [-1.0], [1.0], 8, 2, [[0.0], [2.0]], 1.0, 0), rule=rule)
        s = orc.Solver(p)
        s.build_graph()
        off, tgt, flag, _ = s.graph()
        cnt = np.diff(off)
        assert np.all(flag[1::2] == orc.F_NONFINITE) and np.all(cnt[1::2] == 0)
        assert np.all(flag[0::2] == orc.F_INX) and np.all(cnt[0::2] >= 1)
        assert s.prune() == 8


def test_build_slice_counts_the_slice_edges(orc):
    """The timing slice builds the same pairs as the full graph: its edge count
    equals the full graph's edges of those cells, at level 0 and after a
    refinement."""
    p = dict(W.cstr_256(levels=1, n0=12), rule="outer")
    s = orc.Solver(p)
    nu = len(p["controls"])
    for L in range(2):
        s.build_graph()
        off, _, _, _ = s.graph()
        nl = s.num_live()
        for first, count in ((0, nl), (5, 17), (nl - 3, 10)):
            end = min(nl, first + count)
            assert s.build_slice(first, count) == off[end * nu] - off[first * nu]
        s.build_graph()
        s.prune()
        if L == 0:
            s.subdivide()
