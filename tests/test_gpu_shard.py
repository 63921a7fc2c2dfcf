"""The sharded prune's kernels (gis_shard_*) on one GPU: the graph of a
workload cut into 2 and 3 word-aligned shards, their rounds driven in lock
step with the slices concatenated in-process (the all-gather of a multi-GPU
run), against the oracle's greatest fixed point of the whole graph and
against gis_prune."""
import numpy as np
import pytest

import oracle
from paper_2202_06111_gb300 import workloads as W

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


def _lockstep(shards):
    import torch
    dead, rounds = None, 0
    while True:
        rounds += 1
        gathered = torch.cat([s.round(dead)[0] for s in shards])
        if not bool((gathered != 0).any()):
            return np.concatenate([s.kept() for s in shards]), rounds
        dead = gathered


@pytest.mark.parametrize("world", [1, 2, 3])
@pytest.mark.parametrize("rule", ["outer", "inner"])
def test_shards_match_whole_prune(gis, world, rule):
    from paper_2202_06111_gb300 import shard
    prob = dict(W.cstr_256(levels=0, n0=45), rule=rule)
    with gis.Context(prob) as ctx:
        ctx.build_graph()
        off, tgt, flag = ctx.graph()
        nk, _ = ctx.prune()
        _, fl, _ = ctx.cells()
    n, nu = len(fl), len(prob["controls"])
    parts = shard.partition(n, world)
    shards = [shard.GpuShard(n, f, c, nu, *shard.local_graph(off, tgt, flag, nu, f, c), rule=rule) for f, c in parts]
    kept, rounds = _lockstep(shards)
    for s in shards:
        s.close()
    assert rounds >= 2
    assert np.array_equal(kept, oracle.prune_graph(n, nu, off, tgt, flag, rule=rule))
    assert np.array_equal(kept, (fl & gis.CELL_KEPT) != 0) and kept.sum() == nk


def test_shard_rejects_misaligned_and_bad_graphs(gis):
    import ctypes as C
    L = gis.load()
    h = C.c_void_p()
    off = np.array([0, 1, 2], np.int64)
    tgt = np.array([0, 1], np.int32)
    flag = np.array([1, 1], np.uint8)
    rc = L.gis_shard_create(C.byref(h), 64, 16, 2, 1, off.ctypes.data, tgt.ctypes.data, flag.ctypes.data, 1, None)
    assert rc == gis.EINVAL                          # does not start on a word
    bad = np.array([0, 99], np.int32)
    rc = L.gis_shard_create(C.byref(h), 2, 0, 2, 1, off.ctypes.data, bad.ctypes.data, flag.ctypes.data, 1, None)
    assert rc == gis.EINVAL                          # target out of range
