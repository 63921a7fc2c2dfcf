"""A prune split across processes, one shard per process (one per GPU).

The host side of the sharded fixed point (include/gis.h, gis_shard_*; the
per-process subgraphs and merge of Sec. 3.2 / Fig. 6 applied to the prune of
Sec. 2.3): the cells are cut into contiguous ranges, a shard keeps the
(cell, control) pairs of its cells, and every round each shard's bitmap of
newly removed cells is all-gathered into the round's bitmap of removed cells,
which every shard then applies to its own pairs in its kernels. The loop ends
when a gathered bitmap is empty.

The exchange is any function taking this shard's slice of words and
returning the concatenation of all slices in shard order;
``all_gather_exchange`` does it with torch.distributed (NCCL on GPUs).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import gis

WORD = 32


def partition(n_cells: int, world: int) -> list[tuple[int, int]]:
    """Contiguous (first, count) ranges, one per shard, each starting on a
    multiple of 32 cells and holding a multiple of 32 except the last."""
    words = (n_cells + WORD - 1) // WORD
    out, first = [], 0
    for r in range(world):
        w = words // world + (1 if r < words % world else 0)
        count = min(w * WORD, n_cells - first)
        out.append((first, max(count, 0)))
        first += max(count, 0)
    return out


def local_graph(off, tgt, flag, n_controls: int, first: int, count: int):
    """The shard's pairs: offsets rebased to 0, targets kept global."""
    p0, p1 = first * n_controls, (first + count) * n_controls
    off = np.asarray(off, np.int64)
    loff = np.ascontiguousarray(off[p0:p1 + 1] - off[p0])
    ltgt = np.ascontiguousarray(np.asarray(tgt, np.int32)[off[p0]:off[p1]])
    lflag = np.ascontiguousarray(np.asarray(flag, np.uint8)[p0:p1])
    return loff, ltgt, lflag


class GpuShard:
    """One shard in the library's kernels (gis_shard_*); the bitmaps are
    int32 torch tensors on the current CUDA device."""

    def __init__(self, n_cells_total, first, count, n_controls, off, tgt, flag, rule="outer", stream=None):
        import torch
        L = gis.load()
        self.n_total, self.first, self.count = n_cells_total, first, count
        self._off = np.ascontiguousarray(off, np.int64)
        self._tgt = np.ascontiguousarray(tgt, np.int32)
        self._flag = np.ascontiguousarray(flag, np.uint8)
        h = C.c_void_p()
        st = gis.current_stream() if stream is None else stream
        rc = L.gis_shard_create(C.byref(h), n_cells_total, first, count, n_controls, self._off.ctypes.data,
                                self._tgt.ctypes.data if len(self._tgt) else None, self._flag.ctypes.data,
                                gis.RULES[rule], C.c_void_p(st))
        gis._check(rc)
        self._h = h
        self.out = torch.zeros(max(1, (count + WORD - 1) // WORD), dtype=torch.int32, device="cuda")
        self.started = False

    def round(self, dead):
        """Apply the gathered bitmap of the last round (None for the first);
        returns (this shard's slice of newly removed cells, their number)."""
        n = C.c_int64()
        ptr = None if dead is None else dead.data_ptr()
        gis._check(gis.load().gis_shard_round(self._h, ptr, self.out.data_ptr(), C.byref(n)))
        return self.out[:(self.count + WORD - 1) // WORD], n.value

    def kept(self):
        k = np.zeros(max(self.count, 1), np.uint8)
        n = C.c_int64()
        gis._check(gis.load().gis_shard_kept(self._h, k.ctypes.data, C.byref(n)))
        return k[:self.count].astype(bool)

    def close(self):
        if getattr(self, "_h", None):
            gis.load().gis_shard_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sharded_prune(shard, exchange, max_rounds: int = 1 << 30):
    """Rounds until a gathered bitmap is empty; returns (kept local cells,
    rounds). `shard` has round(dead) -> (slice, n_new) and kept(); `exchange`
    maps this shard's slice to the gathered words of all shards."""
    dead = None
    for rounds in range(1, max_rounds + 1):
        out, _ = shard.round(dead)
        gathered = exchange(out)
        if not bool((gathered != 0).any()):
            return shard.kept(), rounds
        dead = gathered
    raise TimeoutError("sharded prune: round limit reached")


def all_gather_exchange(slices: list[tuple[int, int]], group=None):
    """An exchange over torch.distributed: every rank's slice, padded to the
    longest, all-gathered, then cut back and concatenated in rank order."""
    import torch
    import torch.distributed as dist
    words = [(c + WORD - 1) // WORD for _, c in slices]
    pad = max(max(words), 1)

    def ex(local):
        buf = torch.zeros(pad, dtype=local.dtype, device=local.device)
        buf[:local.numel()] = local
        parts = [torch.empty_like(buf) for _ in slices]
        dist.all_gather(parts, buf, group=group)
        return torch.cat([p[:w] for p, w in zip(parts, words)])

    return ex
