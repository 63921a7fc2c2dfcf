"""Bit-exact kept sets at the workloads' full sizes, against digests of the
FP64 oracle's cell sets written by oracle/write_kept_digests.py (count and
SHA-256 of the sorted (level, idx) rows; tests/golden/kept_digests.json):

  * the 4-D cart-pole workload (48^4 roots, 9 forces, OUTER): the live and
    kept cells of every level the oracle holds in host memory, and the
    covering the next subdivision makes;
  * all 512 instances of the batched workload, solved together by
    gis_batch_solve;
  * a seeded subset of the serving trace (the largest 2-D grids, 48^4 and
    24^4 cart-pole requests) served by continuous batching beside other
    requests."""
import json
import os

import pytest

from paper_2202_06111_gb300 import workloads as W

from gis_compare import digest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "kept_digests.json")


@pytest.fixture(scope="module")
def gis():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2202_06111_gb300 import build, gis as g
    build.build()
    g.load()
    return g


@pytest.fixture(scope="module")
def golden():
    return json.load(open(GOLDEN))


def _same(got, want, what):
    assert got["count"] == want["count"], f"{what}: {got['count']} cells on the GPU vs {want['count']} (oracle)"
    assert got["sha256"] == want["sha256"], f"{what}: same count, different cells"


def test_cartpole_48_levels(gis, golden):
    g = golden["cartpole_48"]
    prob = dict(W.cartpole_48(), rule="outer")
    assert g["problem"]["n0"] == prob["n0"] and g["problem"]["rule"] == "outer"
    with gis.Context(prob) as ctx:
        for rec in g["levels"]:
            L = rec["level"]
            ctx.build_graph()
            lv, fl, idx = ctx.cells()
            _same(digest(lv, idx), rec["live"], f"level {L} live cells")
            nk, _ = ctx.prune()
            assert nk == rec["kept"]["count"], f"level {L}: kept {nk} vs {rec['kept']['count']}"
            _same(digest(*ctx.kept_cells()), rec["kept"], f"level {L} kept cells")
            ctx.subdivide()
        nxt = g["next_covering"]
        ctx.build_graph()
        lv, fl, idx = ctx.cells()
        _same(digest(lv, idx), nxt["live"], f"level {nxt['level']} covering")


def test_batch_512_all_instances(gis, golden):
    want = golden["batch_512"]["instances"]
    probs = W.batch_512()
    assert len(want) == len(probs) == 512
    for p, w in zip(probs, want):
        assert w["problem"]["name"] == p["name"]
        p["cells_cap"] = max(1, w["kept"]["count"])
    res, stats = gis.batch_solve(probs)
    bad = []
    for p, r, w in zip(probs, res, want):
        assert r["status"] == 0 and r["levels_done"] == p["levels"], p["name"]
        if r["n_kept"] != w["kept"]["count"] or r["n_cells"] != w["n_cells"] or digest(*r["kept"]) != w["kept"]:
            bad.append(p["name"])
    assert not bad, f"{len(bad)} of 512 instances differ from the oracle, e.g. {bad[:5]}"


def test_serving_subset(gis, golden):
    want = {r["request_id"]: r for r in golden["serving"]["requests"]}
    trace = W.serving_2000()
    subset = [trace[i] for i in sorted(want)]
    others = [r for r in trace[:40] if r["request_id"] not in want and r["n"] == 2]
    srv = gis.Server()
    tickets = {}
    for j, r in enumerate(subset):               # the recorded requests among others
        for o in others[4 * j:4 * j + 4]:
            tickets[srv.submit(o)] = None
        r = dict(r, cells_cap=max(1, want[r["request_id"]]["kept"]["count"]))
        tickets[srv.submit(r)] = r["request_id"]
    got = {}
    for t, rid in tickets.items():
        res = srv.poll(t, wait=True, want_cells=rid is not None)
        assert res["status"] == 0
        if rid is not None:
            got[rid] = res
    st = srv.stats()
    srv.close()
    assert st["failed"] == 0
    for rid, w in want.items():
        r = got[rid]
        assert r["n_cells"] == w["n_cells"], rid
        _same(digest(*r["kept"]), w["kept"], f"request {rid} ({w['problem']['name']})")
