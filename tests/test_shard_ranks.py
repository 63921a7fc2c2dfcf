"""The sharded prune's host loop (paper_2202_06111_gb300/shard.py) on two gloo
ranks on the CPU: the partition into word-aligned cell ranges, the per-round
all-gather of the removed-cell bitmaps and the end of the rounds, checked
against the oracle's greatest fixed point of the whole graph. Each rank's
local round is a numpy stand-in with the semantics of the library's shard
kernels (those run on the GPU in test_gpu_shard.py)."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class NumpyShard:
    """A shard's rounds: INNER / OUTER pair budgets, viable pairs per cell,
    the pairs referring to each global cell."""

    def __init__(self, n_total, first, count, nu, off, tgt, flag, rule):
        self.count, self.nu, self.rule = count, nu, rule
        P = count * nu
        if rule == "outer":
            self.budget = np.diff(off).astype(np.int64)
        else:
            ok = ((flag & 1) != 0) & ((flag & 6) == 0)
            self.budget = ok.astype(np.int64)
        self.viable = (self.budget.reshape(count, nu) > 0).sum(axis=1) if count else np.zeros(0, np.int64)
        self.kept_ = self.viable > 0
        self.refs = [[] for _ in range(n_total)]
        for p in range(P):
            for e in range(off[p], off[p + 1]):
                self.refs[tgt[e]].append(p)
        self.started = False

    def _slice(self, dead_local):
        words = np.zeros(max(1, (self.count + 31) // 32), np.uint32)
        for i in np.nonzero(dead_local)[0]:
            words[i >> 5] |= np.uint32(1 << (i & 31))
        return torch.from_numpy(words[:(self.count + 31) // 32].view(np.int32).copy())

    def round(self, dead):
        newly = np.zeros(self.count, bool)
        if not self.started:
            self.started = True
            newly = ~self.kept_
        else:
            bits = np.unpackbits(dead.numpy().view(np.uint8), bitorder="little")
            for j in np.nonzero(bits)[0]:
                for p in self.refs[j]:
                    if self.budget[p] <= 0:
                        continue
                    self.budget[p] = self.budget[p] - 1 if self.rule == "outer" else 0
                    if self.budget[p] == 0:
                        i = p // self.nu
                        self.viable[i] -= 1
                        if self.viable[i] == 0:
                            self.kept_[i] = False
                            newly[i] = True
        return self._slice(newly), int(newly.sum())

    def kept(self):
        return self.kept_.copy()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _graph(rule):
    import oracle
    from paper_2202_06111_gb300 import workloads as W
    s = oracle.Solver(dict(W.cstr_256(levels=0, n0=21), rule=rule))
    s.build_graph()
    off, tgt, flag, _ = s.graph()
    return s.num_live(), len(W.cstr_256()["controls"]), off, tgt, flag


def _rank(rank, ws, port, rule, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    from paper_2202_06111_gb300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        n, nu, off, tgt, flag = _graph(rule)
        parts = shard.partition(n, ws)
        first, count = parts[rank]
        loff, ltgt, lflag = shard.local_graph(off, tgt, flag, nu, first, count)
        sh = NumpyShard(n, first, count, nu, loff, ltgt, lflag, rule)
        kept, rounds = shard.sharded_prune(sh, shard.all_gather_exchange(parts))
        out[rank] = (first, kept.tolist(), rounds)
    finally:
        dist.destroy_process_group()


def test_partition_is_word_aligned():
    sys.path.insert(0, ROOT)
    from paper_2202_06111_gb300 import shard
    for n, w in ((441, 2), (1000, 3), (64, 4), (31, 2), (0, 2)):
        parts = shard.partition(n, w)
        assert sum(c for _, c in parts) == n and len(parts) == w
        for r, (f, c) in enumerate(parts):
            assert f % 32 == 0 or c == 0              # an empty shard may sit at the end
            assert c % 32 == 0 or f + c == n


@pytest.mark.parametrize("rule", ["outer", "inner"])
def test_sharded_prune_two_ranks(rule):
    import oracle
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, rule, out)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    n, nu, off, tgt, flag = _graph(rule)
    want = oracle.prune_graph(n, nu, off, tgt, flag, rule=rule)
    got = np.zeros(n, bool)
    rounds = set()
    for r in range(ws):
        first, kept, rd = out[r]
        got[first:first + len(kept)] = kept
        rounds.add(rd)
    assert len(rounds) == 1                          # every rank saw the same empty round
    assert np.array_equal(got, want)
    assert 0 < want.sum() < n                        # a non-trivial fixed point
