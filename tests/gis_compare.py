"""Helpers that compare GPU results with the oracle, element by element.

Cells are matched by their key (level, idx); pairs by (cell, control); targets
are remapped to the oracle's canonical cell order and compared as sorted lists.
"""
import numpy as np


def keys(level, idx):
    return np.concatenate([np.asarray(level, np.int64)[:, None], np.asarray(idx, np.int64)], axis=1)


def perm_to_oracle(gpu_level, gpu_idx, orc_level, orc_idx):
    """perm[g] = oracle slot of GPU slot g; asserts both hold the same cells."""
    gk, ok = keys(gpu_level, gpu_idx), keys(orc_level, orc_idx)
    assert gk.shape == ok.shape, f"{len(gk)} live cells on the GPU vs {len(ok)} in the oracle"
    go = np.lexsort(gk.T[::-1])
    oo = np.lexsort(ok.T[::-1])
    assert np.array_equal(gk[go], ok[oo]), "live cell sets differ"
    perm = np.empty(len(gk), np.int64)
    perm[go] = oo
    return perm


def canonical_edges(off, tgt, nu, perm=None):
    """(pair, target) rows sorted, with cells renumbered by perm."""
    P = len(off) - 1
    cnt = np.diff(off)
    pair = np.repeat(np.arange(P, dtype=np.int64), cnt)
    t = np.asarray(tgt, np.int64)
    if perm is not None:
        pair = perm[pair // nu] * nu + pair % nu
        t = perm[t]
    o = np.lexsort((t, pair))
    return pair[o], t[o]


def compare_graph(gpu_graph, orc_graph, perm, nu, flag_mask=7):
    goff, gtgt, gflag = gpu_graph
    ooff, otgt, oflag, _ = orc_graph
    gp, gt = canonical_edges(goff, gtgt, nu, perm)
    op, ot = canonical_edges(ooff, otgt, nu, None)
    P = len(ooff) - 1
    gf = np.empty(P, np.uint8)
    pidx = np.arange(P)
    gf[perm[pidx // nu] * nu + pidx % nu] = gflag & flag_mask
    bad_flags = np.nonzero(gf != (oflag & flag_mask))[0]
    same_edges = len(gp) == len(op) and np.array_equal(gp, op) and np.array_equal(gt, ot)
    return same_edges, bad_flags, (len(gp), len(op))


def first_edge_diff(gpu_graph, orc_graph, perm, nu):
    goff, gtgt, _ = gpu_graph
    ooff, otgt, _, _ = orc_graph
    gp, gt = canonical_edges(goff, gtgt, nu, perm)
    op, ot = canonical_edges(ooff, otgt, nu, None)
    gs = set(zip(gp.tolist(), gt.tolist()))
    os_ = set(zip(op.tolist(), ot.tolist()))
    only_g = sorted(gs - os_)[:5]
    only_o = sorted(os_ - gs)[:5]
    return only_g, only_o


def kept_keys(level, idx):
    k = keys(level, idx)
    return set(map(tuple, k.tolist()))


def digest(level, idx):
    """Count and SHA-256 of a cell set: rows (level, idx_0..idx_{n-1}) as
    little-endian int32, sorted lexicographically (the form of the stored
    oracle digests in tests/golden/kept_digests.json)."""
    import hashlib
    rows = keys(level, idx)
    rows = rows[np.lexsort(rows.T[::-1])] if len(rows) else rows
    return {"count": int(len(rows)), "sha256": hashlib.sha256(rows.astype("<i4").tobytes()).hexdigest()}
