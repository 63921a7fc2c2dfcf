"""Write tests/golden/kept_digests.json: the FP64 oracle's kept cell sets of the
full-size workloads, as digests, for the GPU parity tests.

TEST INFRASTRUCTURE: calls only the oracle (and the seeded problem
definitions); nothing here comes from the CUDA path.

A cell set is written as its count and the SHA-256 of its canonical form:
rows (level, idx_0 .. idx_{n-1}) as little-endian int32, sorted
lexicographically, concatenated. What is recorded:

  cartpole_48   the 4-D cart-pole workload (48^4 roots, 9 forces, OUTER, the
                rule the benchmark runs): per level the live cells and the kept
                cells (Sec. 2.3), for every level whose graph fits in this
                host's memory, and the covering of the next level (the live
                cells after the boundary subdivision of Sec. 3.1).
  batch_512     every one of the 512 uneven instances: its kept cells after
                its last level.
  serving       a seeded subset of the 2000 serving requests: the largest
                2-D grids (about 1000^2 roots, 0-3 levels) and cart-pole
                requests, among them full 48^4 grids.

  python oracle/write_kept_digests.py [--only cartpole_48,batch_512,serving]
        [--cartpole-levels 2] [--threads 0]

Each part merges into the existing file, so parts may be run separately.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2202_06111_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(ROOT, "tests", "golden", "kept_digests.json")

# serving requests whose oracle solves are recorded (seeded trace order)
SERVING_2D_LARGEST = 8
SERVING_CARTPOLE = 6


def digest(level, idx) -> dict:
    rows = np.concatenate([np.asarray(level, np.int64)[:, None], np.asarray(idx, np.int64)], axis=1)
    rows = rows[np.lexsort(rows.T[::-1])] if len(rows) else rows
    return {"count": int(len(rows)), "sha256": hashlib.sha256(rows.astype("<i4").tobytes()).hexdigest()}


def _problem_key(p: dict) -> dict:
    return {k: p[k] for k in ("name", "dyn", "n0", "levels", "rule") if k in p}


def cartpole_48(levels: int) -> dict:
    """Level by level: live and kept cells of levels 0 .. levels-1, and the live
    cells of level `levels` (the covering after the last recorded split)."""
    prob = dict(W.cartpole_48(), rule="outer")
    s = oracle.Solver(prob)
    rec = {"problem": _problem_key(prob), "levels": []}
    for L in range(levels):
        t = time.time()
        s.build_graph()
        lv, idx = s.live()
        live = digest(lv, idx)
        nk = s.prune()
        kl, ki = s.kept_cells()
        kept = digest(kl, ki)
        assert kept["count"] == nk
        rec["levels"].append({"level": L, "live": live, "kept": kept, "edges": int(s.num_edges())})
        print(f"cartpole_48 L{L}: live {live['count']} kept {nk} ({time.time() - t:.0f} s)", flush=True)
        s.subdivide()
    # the covering of the next level: its live cells, numbered by a graph
    # build would need that level's whole graph, so they are read from the tree
    lv, st, idx, ch = s.nodes()
    alive = st == oracle.ALIVE
    rec["next_covering"] = {"level": levels, "live": digest(lv[alive], idx[alive])}
    print(f"cartpole_48 L{levels} covering: {int(alive.sum())} live cells", flush=True)
    return rec


def batch_512() -> dict:
    out = []
    t = time.time()
    for i, p in enumerate(W.batch_512()):
        s = oracle.solve(p)
        kl, ki = s.kept_cells()
        out.append({"problem": _problem_key(p), "n_cells": int(s.num_live()), "kept": digest(kl, ki)})
        if i % 64 == 63:
            print(f"batch_512: {i + 1} instances ({time.time() - t:.0f} s)", flush=True)
    return {"instances": out}


def serving_subset() -> list[int]:
    """Request ids of the recorded subset: the largest 2-D grids, and the
    cart-pole requests of the full 48^4 grid at level 0 plus the largest
    whose three levels the oracle solves in minutes (n0 <= 24)."""
    reqs = W.serving_2000()
    two = sorted((r for r in reqs if r["n"] == 2), key=lambda r: (r["n0"][0] * r["n0"][1], r["request_id"]))
    ids = [r["request_id"] for r in two[-SERVING_2D_LARGEST:]]
    cp = [r for r in reqs if r["dyn"] == "cartpole"]
    full = [r["request_id"] for r in cp if r["n0"][0] == 48 and r["levels"] == 0]
    deep = sorted((r for r in cp if r["n0"][0] <= 24 and r["levels"] == 3),
                  key=lambda r: (r["n0"][0], r["request_id"]))
    ids += full[:2] + [r["request_id"] for r in deep[-(SERVING_CARTPOLE - len(full[:2])):]]
    return sorted(ids)


def serving() -> dict:
    reqs = {r["request_id"]: r for r in W.serving_2000()}
    out = []
    t = time.time()
    for i in serving_subset():
        p = reqs[i]
        s = oracle.solve(p)
        kl, ki = s.kept_cells()
        out.append({"request_id": i, "problem": _problem_key(p), "n_cells": int(s.num_live()),
                    "kept": digest(kl, ki)})
        print(f"serving request {i} ({p['name']}, {p['levels']} levels): kept {len(kl)} "
              f"({time.time() - t:.0f} s)", flush=True)
    return {"requests": out}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", default="cartpole_48,batch_512,serving")
    ap.add_argument("--cartpole-levels", type=int, default=2)
    ap.add_argument("--threads", type=int, default=0)
    a = ap.parse_args()
    oracle.build()
    threads = oracle.set_threads(a.threads)
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    data["_format"] = ("count and SHA-256 of the sorted rows (level, idx_0..idx_{n-1}) as little-endian int32; "
                       "written by oracle/write_kept_digests.py from the FP64 oracle")
    for part in a.only.split(","):
        t = time.time()
        if part == "cartpole_48":
            data[part] = cartpole_48(a.cartpole_levels)
        elif part == "batch_512":
            data[part] = batch_512()
        elif part == "serving":
            data[part] = serving()
        else:
            raise SystemExit(f"unknown part {part}")
        data[part]["oracle_seconds"] = round(time.time() - t, 1)
        data[part]["oracle_threads"] = threads
        json.dump(data, open(OUT, "w"), indent=1)
        print(f"{part}: written ({time.time() - t:.0f} s)", flush=True)


if __name__ == "__main__":
    main()
