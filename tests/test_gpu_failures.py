"""Failure paths on the GPU, made without faulting it. A prune whose round
limit runs out returns GIS_ETIMEOUT (the bounded frontier loop gives up and
reports) and the device stays usable; a device allocation that fails inside a
served step (injected on the host by the GIS_TEST_FAIL_ALLOC hook) makes the
server re-queue that step's requests to run alone, and every result still
equals the oracle's."""
import pytest

import oracle
from paper_2202_06111_gb300 import workloads as W

from gis_compare import kept_keys
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
def test_prune_round_limit_times_out(gis, rule):
    prob = dict(W.cstr_256(levels=0, n0=64), rule=rule)
    with gis.Context(prob) as ctx:
        ctx.build_graph()
        _, rounds = ctx.prune()
    assert rounds >= 3
    with gis.Context(prob, round_limit=1) as ctx:
        ctx.build_graph()
        with pytest.raises(gis.GisError) as e:
            ctx.prune()
        assert e.value.status == gis.ETIMEOUT
    # the device and the library are still usable, and right
    run_both(gis, prob, 0)


def test_server_requeues_a_step_that_runs_out_of_memory(gis, monkeypatch):
    monkeypatch.setenv("GIS_TEST_FAIL_ALLOC", "7")
    reqs = [dict(W.cstr_256(levels=2, n0=24), rule="outer"), W.vdp_64(n0=24), W.cstr_256(levels=1, n0=20),
            dict(W.cartpole_48(levels=1, n0=5), rule="outer")]
    srv = gis.Server(max_active=8)
    tickets = [srv.submit(r) for r in reqs]
    results = [srv.poll(t, wait=True) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["oom_restarts"] == 1 and st["failed"] == 0 and st["completed"] == len(reqs)
    for r, res in zip(reqs, results):
        assert res["status"] == 0 and res["levels_done"] == r["levels"]
        assert kept_keys(*res["kept"]) == kept_keys(*oracle.solve(r).kept_cells()), r["name"]
