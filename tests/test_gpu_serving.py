"""Serving by continuous batching: requests submitted while others run are
admitted at the next step and share its launches; every result equals the
request solved alone (GPU context) and the oracle's."""
import time

import numpy as np
import pytest

import oracle
from paper_2202_06111_gb300 import workloads as W

from gis_compare import kept_keys

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


def _mix(count=30):
    reqs = W.serving_2000(count=count, max_2d_cells=80.0 ** 2, max_4d_n0=10.0)
    for r in reqs:
        if r["dyn"] == "cartpole":
            r["levels"] = min(r["levels"], 1)
            r["rule"] = "outer"
    return reqs


def test_serving_results_equal_alone_and_oracle(gis):
    reqs = _mix()
    srv = gis.Server(max_active=8)
    tickets = []
    for i, r in enumerate(reqs):          # staggered: later requests join running steps
        tickets.append(srv.submit(r))
        if i % 5 == 4:
            time.sleep(0.02)
    results = [srv.poll(t, wait=True) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["steps"] > max(r["levels"] for r in reqs) + 1       # requests joined over several steps
    for r, res in zip(reqs, results):
        assert res["status"] == 0 and res["levels_done"] == r["levels"]
        with gis.Context(r) as ctx:
            ctx.solve()
            alone = kept_keys(*ctx.kept_cells())
        served = kept_keys(*res["kept"])
        assert served == alone, r["name"]
        ref = oracle.solve(r)
        assert served == kept_keys(*ref.kept_cells()), r["name"]


def test_serving_admission_by_memory(gis):
    """With a budget below two requests' estimate the server admits one at a
    time and still completes all of them."""
    reqs = [W.cstr_256(levels=1, n0=32), W.vdp_64(n0=32), W.cstr_256(levels=2, n0=24)]
    srv = gis.Server(max_device_bytes=1)
    ts = [srv.submit(r) for r in reqs]
    res = [srv.poll(t, wait=True) for t in ts]
    st = srv.stats()
    srv.close()
    assert all(r["status"] == 0 for r in res) and st["completed"] == 3
    assert st["steps"] >= sum(r["levels"] + 1 for r in reqs)     # one request per step


def test_serving_rejects_bad_request(gis):
    srv = gis.Server()
    bad = dict(W.vdp_64(), n0=[0, 4])
    with pytest.raises(gis.GisError):
        srv.submit(bad)
    srv.close()
