"""gis_prune_graph_noalloc: pruning without any device allocation.

Some callers cannot allocate device memory (a fixed memory arena, an
allocator that owns the device, paths that must not synchronise). This entry
point prunes a graph they pass in, with its scratch in a fixed array of the
library. Checked through the C ABI against gis_prune and against the oracle's
greatest fixed point (Sec. 2.3) on the same graphs, on several calls in a row
(the shared scratch keeps the previous call's contents), and for the size
limits."""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2202_06111_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2202_06111_gb300 import build, gis
    build.build()
    return gis


def _graph_and_kept(gis, prob):
    ctx = gis.Context(prob)
    ctx.build_graph()
    off, tgt, flag = ctx.graph()
    ctx.prune()
    lv, fl, idx = ctx.cells()
    ctx.close()
    return off, tgt, flag, ((fl & gis.CELL_KEPT) != 0).astype(np.uint8)


def _noalloc(gis, off, tgt, flag, n_cells, nu, rule):
    import torch
    d_off = torch.from_numpy(off).cuda()
    d_tgt = torch.from_numpy(tgt.astype(np.int32)).cuda() if len(tgt) else torch.zeros(1, dtype=torch.int32).cuda()
    d_flag = torch.from_numpy(flag).cuda()
    kept = torch.full((max(n_cells, 1),), 7, dtype=torch.uint8, device="cuda")   # garbage in, must be overwritten
    nk = C.c_int64(-1)
    st = torch.cuda.current_stream()
    rc = gis.load().gis_prune_graph_noalloc(n_cells, nu, d_off.data_ptr(), d_tgt.data_ptr(), d_flag.data_ptr(),
                                            len(tgt), gis.RULES[rule], kept.data_ptr(), C.byref(nk),
                                            C.c_void_p(st.cuda_stream))
    return rc, kept[:n_cells].cpu().numpy(), nk.value


def test_noalloc_prune_matches_gis_prune(lib):
    gis = lib
    cases = [(dict(W.cstr_256(levels=0, n0=64), rule="inner"), "inner"),
             (dict(W.cstr_256(levels=0, n0=48), rule="outer"), "outer"),
             (dict(W.vdp_64(), rule="outer"), "outer")]
    graphs = [(_graph_and_kept(gis, p), p, r) for p, r in cases]
    # several calls in a row, sizes going down and up again
    for (off, tgt, flag, kept_ref), prob, rule in graphs + graphs[:1]:
        n_cells = len(kept_ref)
        nu = len(prob["controls"])
        rc, kept, nk = _noalloc(gis, off, tgt, flag, n_cells, nu, rule)
        assert rc == gis.OK, gis.load().gis_last_error(None)
        assert np.array_equal(kept, kept_ref)
        assert nk == int(kept_ref.sum())
        # the oracle's fixed point on the same CSR
        want = oracle.prune_graph(n_cells, nu, off, tgt, flag, rule=rule)
        assert np.array_equal(kept.astype(bool), want)


def test_noalloc_rejects_oversize_and_bad_graphs(lib):
    gis = lib
    L = gis.load()
    big = 1 << 18
    rc = L.gis_prune_graph_noalloc(big, 1, None, None, None, 0, 0, None, None, None)
    assert rc == gis.EUNSUPPORTED
    assert b"exceed" in L.gis_last_error(None)
    # factors whose product would overflow int64 are rejected, not multiplied
    rc = L.gis_prune_graph_noalloc((1 << 62) - 1, 4, None, None, None, 0, 0, None, None, None)
    assert rc == gis.EUNSUPPORTED
    rc = L.gis_prune_graph_noalloc(2, (1 << 31) - 1, None, None, None, 0, 0, None, None, None)
    assert rc == gis.EUNSUPPORTED
    off = np.array([0, 1, 2], np.int64)
    tgt = np.array([0, 5], np.int32)                 # 5 is not a cell of a 2-cell graph
    flag = np.array([1, 1], np.uint8)
    rc, _, _ = _noalloc(gis, off, tgt, flag, 2, 1, "inner")
    assert rc == gis.EINVAL
    # the scratch is intact afterwards
    off, tgt, flag, kept_ref = _graph_and_kept(gis, dict(W.vdp_64(n0=16), rule="inner"))
    rc, kept, _ = _noalloc(gis, off, tgt, flag, len(kept_ref), 5, "inner")
    assert rc == gis.OK and np.array_equal(kept, kept_ref)
