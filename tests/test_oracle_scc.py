"""Pins of the oracle's literal Def. 3 rule ("scc"): the largest strongly
connected component of the cell graph plus every cell with a path into it
(readings: a component needs a cycle; ties keep every largest component).
Hand-built graphs, a library routine (networkx) on random graphs, and the
inclusion in the OUTER fixed point on a real problem."""
import numpy as np
import pytest

from paper_2202_06111_gb300 import workloads as W


def _csr(n, n_u, edges):
    """edges: (cell, control, target) -> pair CSR (off, tgt, flag)."""
    per = [[[] for _ in range(n_u)] for _ in range(n)]
    for i, u, j in edges:
        per[i][u].append(j)
    off, tgt = [0], []
    for i in range(n):
        for u in range(n_u):
            tgt += sorted(set(per[i][u]))
            off.append(len(tgt))
    return np.array(off, np.int64), np.array(tgt or [0], np.int32)[:len(tgt)], np.ones(n * n_u, np.uint8)


def _scc(orc, n, n_u, edges):
    off, tgt, flag = _csr(n, n_u, edges)
    return orc.prune_graph(n, n_u, off, tgt, flag, rule="scc")


def test_cycle_dag_selfloop(orc):
    assert _scc(orc, 4, 1, [(0, 0, 1), (1, 0, 2), (2, 0, 3), (3, 0, 0)]).all()
    assert not _scc(orc, 4, 1, [(0, 0, 1), (1, 0, 2), (2, 0, 3)]).any()          # no cycle: nothing
    k = _scc(orc, 3, 1, [(0, 0, 1), (1, 0, 1), (2, 0, 0)])                      # self-loop on 1
    assert k.tolist() == [True, True, True]


def test_largest_component_and_ancestors(orc):
    # a 3-cycle {0,1,2}, a 5-cycle {3..7}, 8 -> 3 (ancestor of the 5-cycle),
    # 9 -> 0 (ancestor of the small one), 7 -> 10 (a descendant: dropped)
    e = [(0, 0, 1), (1, 0, 2), (2, 0, 0), (3, 1, 4), (4, 0, 5), (5, 1, 6), (6, 0, 7), (7, 1, 3),
         (8, 0, 3), (9, 1, 0), (7, 0, 10)]
    k = _scc(orc, 11, 2, e)
    assert np.flatnonzero(k).tolist() == [3, 4, 5, 6, 7, 8]


def test_ties_keep_every_largest(orc):
    e = [(0, 0, 1), (1, 0, 0), (2, 0, 3), (3, 0, 2), (4, 0, 0), (4, 0, 2)]
    assert _scc(orc, 5, 1, e).all()


def test_random_graphs_against_networkx(orc):
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(11)
    for trial in range(300):
        n = int(rng.integers(1, 40))
        n_u = int(rng.integers(1, 4))
        m = int(rng.integers(0, 3 * n))
        edges = [(int(rng.integers(n)), int(rng.integers(n_u)), int(rng.integers(n))) for _ in range(m)]
        got = _scc(orc, n, n_u, edges)
        G = nx.DiGraph()
        G.add_nodes_from(range(n))
        G.add_edges_from((i, j) for i, _, j in edges)
        comps = [c for c in nx.strongly_connected_components(G) if len(c) > 1 or G.has_edge(next(iter(c)),
                                                                                             next(iter(c)))]
        want = np.zeros(n, bool)
        if comps:
            best = max(len(c) for c in comps)
            keep = set().union(*[c for c in comps if len(c) == best])
            for c in list(keep):
                keep |= nx.ancestors(G, c)
            want[list(keep)] = True
        assert np.array_equal(got, want), (trial, n, n_u, edges)


def test_scc_inside_outer_fixed_point(orc):
    """A cell with a path into a cycle has an infinite path, so the literal rule
    keeps a subset of the OUTER greatest fixed point."""
    base = W.problem(W.vdp(1.0), [-3, -3], [3, 3], 10, 3, W.controls_grid(-1, 1, 3), 0.25, 2, precision="fp64")
    ks = {}
    for rule in ("scc", "outer"):
        s = orc.Solver(dict(base, rule=rule))
        s.build_graph()
        s.prune()
        ks[rule] = s.kept()
    assert ks["scc"].sum() > 0
    assert np.all(~ks["scc"] | ks["outer"])
