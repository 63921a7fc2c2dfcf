"""Parity at the workloads' full sizes: every edge and kept cell of the CSTR
workload (256^2 roots, 3 levels) in both rules; the 4-D cart-pole workload's
level-0 graph (48^4 roots, 9 forces, 771M edges) by per-pair counts and flags
for every pair and exact targets for a random sample of pairs; and the
batched API against one oracle solve per problem."""
import numpy as np
import pytest

import oracle
from paper_2202_06111_gb300 import workloads as W

from gis_compare import kept_keys, perm_to_oracle
from test_gpu_parity import run_both

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gis():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2202_06111_gb300 import build, gis as g
    build.build()
    g.load()
    oracle.build()
    oracle.set_threads(0)
    return g


@pytest.mark.parametrize("rule", ["inner", "outer"])
def test_cstr_256_full(gis, rule):
    run_both(gis, dict(W.cstr_256(), rule=rule), 3)


def test_cartpole_48_level0_full(gis):
    prob = dict(W.cartpole_48(), rule="inner")
    ctx = gis.Context(prob)
    ctx.build_graph()
    ref = oracle.Solver(prob)
    ref.build_graph()
    glv, _, gidx = ctx.cells()
    olv, oidx = ref.live()
    perm = perm_to_oracle(glv, gidx, olv, oidx)
    nu = len(prob["controls"])
    goff, gtgt, gflag = ctx.graph()
    ooff, otgt, oflag, _ = ref.graph()
    P = len(oflag)
    pidx = np.arange(P)
    q = perm[pidx // nu] * nu + pidx % nu          # GPU pair -> oracle pair
    assert np.array_equal(np.diff(goff), np.diff(ooff)[q]), "per-pair target counts differ"
    assert np.array_equal(gflag & 7, (oflag & 7)[q]), "pair flags differ"
    rng = np.random.default_rng(7)
    inv = np.empty(len(perm), np.int64)
    inv[perm] = np.arange(len(perm))
    for p in rng.choice(P, 200000, replace=False):
        g = np.sort(perm[gtgt[goff[p]:goff[p + 1]]])
        o = otgt[ooff[q[p]]:ooff[q[p] + 1]]
        assert np.array_equal(g, o), p
    nk, _ = ctx.prune()
    assert nk == ref.prune()
    ctx.close()


def test_cartpole_outer_two_levels(gis):
    run_both(gis, dict(W.cartpole_48(levels=2, n0=12), rule="outer"), 2)


def test_batch_matches_single_solves(gis):
    """gis_batch_solve over uneven problems (different systems, grids, controls
    and depths in the same launches) equals one oracle solve per problem."""
    probs = W.batch_512(count=24, max_cells=96.0 ** 2)
    res, stats = gis.batch_solve(probs)
    assert stats["cum_cells_built"] == sum(r["cells_built"] for r in res)
    for p, r in zip(probs, res):
        s = oracle.solve(p)
        olv, oidx = s.kept_cells()
        assert r["status"] == 0 and r["levels_done"] == p["levels"]
        assert r["n_kept"] == len(olv), p["name"]
        assert kept_keys(*r["kept"]) == kept_keys(olv, oidx), p["name"]
