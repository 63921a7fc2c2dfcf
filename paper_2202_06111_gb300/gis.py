"""ctypes binding of libgis (include/gis.h): argument marshalling only.

Every computation runs in the CUDA kernels of libgis.so. There is no CPU
fallback: if the library cannot be loaded, or no GPU is present, the calls
raise.

The C entry points keep their names (``gis_create``, ``gis_build_graph``,
``gis_prune``, ``gis_subdivide``, ``gis_solve``, ``gis_get_cells``,
``gis_get_graph``, ``gis_get_boxes``, ``gis_get_stats``, ``gis_batch_solve``);
``Context`` and ``batch_solve`` wrap them for problems given as the dicts of
``paper_2202_06111_gb300.workloads``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgis.so")

MAXN, NPARAM = 4, 32
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED, ECANCELLED, EBOUNDS, ESTATE = 0, -1, -2, -3, -4, -5, -6, -7, -8
DYN_IDS = {"linmap": 0, "vdp": 1, "cstr_dl": 2, "cartpole": 3, "cstr_paper": 4}
RULES = {"inner": 0, "outer": 1, "scc": 2}
PRECISIONS = {"fp64": 0, "fp32": 1}
ENCLOSURES = {"samples": 0, "interval": 1}
SPLITS = {"all": 0, "cycled": 1}
PAIR_INX, PAIR_TOUCH_DEAD, PAIR_NONFINITE = 1, 2, 4
CELL_KEPT, CELL_BOUNDARY = 1, 2


class GisError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libgis status {status}: {msg}")
        self.status = status


class gis_dynamics(C.Structure):
    _fields_ = [("dyn_id", C.c_int32), ("n", C.c_int32), ("m", C.c_int32), ("substeps", C.c_int32),
                ("dt", C.c_double), ("params", C.c_double * NPARAM)]


class gis_grid(C.Structure):
    _fields_ = [("lo", C.c_double * MAXN), ("hi", C.c_double * MAXN), ("root_cells", C.c_int32 * MAXN),
                ("k_samples", C.c_int32)]


class gis_controls(C.Structure):
    _fields_ = [("n_controls", C.c_int32), ("u", C.POINTER(C.c_double))]


class gis_options(C.Structure):
    _fields_ = [("rule", C.c_int32), ("precision", C.c_int32), ("band", C.c_double),
                ("lanes_per_pair", C.c_int32), ("timing", C.c_int32), ("max_device_bytes", C.c_int64),
                ("round_limit", C.c_int64), ("enclosure_store", C.c_int32), ("fixed_shapes", C.c_int32),
                ("split_ring", C.c_int32), ("enclosure", C.c_int32), ("split", C.c_int32),
                ("reserved", C.c_int32)]


class gis_cell(C.Structure):
    _fields_ = [("level", C.c_int32), ("flags", C.c_int32), ("idx", C.c_int32 * MAXN)]


_STAT_FIELDS = [("finest_level", C.c_int32), ("level", C.c_int32), ("n_nodes", C.c_int64), ("n_live", C.c_int64),
                ("n_pairs", C.c_int64), ("n_edges", C.c_int64), ("n_kept", C.c_int64), ("n_split", C.c_int64),
                ("n_new_pairs", C.c_int64), ("n_recheck", C.c_int64), ("prune_rounds", C.c_int32),
                ("lanes_per_pair", C.c_int32), ("cum_cells_built", C.c_int64), ("cum_pairs_propagated", C.c_int64),
                ("cum_edges", C.c_int64), ("cum_recheck", C.c_int64), ("cum_prop_launches", C.c_int64),
                ("ms_prop", C.c_double), ("ms_bin", C.c_double), ("ms_recheck", C.c_double),
                ("ms_count", C.c_double), ("ms_scan", C.c_double), ("ms_fill", C.c_double),
                ("ms_transpose", C.c_double), ("ms_prune", C.c_double), ("ms_classify", C.c_double),
                ("ms_split", C.c_double), ("ms_other", C.c_double), ("prop_flops", C.c_double),
                ("graph_bytes", C.c_double), ("prune_bytes", C.c_double), ("count_bytes", C.c_double),
                ("fill_bytes", C.c_double), ("transpose_bytes", C.c_double), ("cum_launches", C.c_int64),
                ("cum_recheck_samples", C.c_int64), ("n_cell_edges", C.c_int64), ("cum_cell_edges", C.c_int64),
                ("cum_recheck_fp64", C.c_int64), ("lattice_tile_cells", C.c_int32),
                ("sibling_parents", C.c_int32), ("cum_tune_launches", C.c_int64), ("stage_cap", C.c_int64),
                ("stage_edges", C.c_int64), ("stage_lost_chunks", C.c_int64), ("free_bytes_at_stage", C.c_int64),
                ("scc_passes", C.c_int64)]


class gis_stats(C.Structure):
    _fields_ = _STAT_FIELDS


class gis_request(C.Structure):
    _fields_ = [("dyn", gis_dynamics), ("grid", gis_grid), ("controls", gis_controls), ("levels", C.c_int32),
                ("rule", C.c_int32), ("precision", C.c_int32), ("band", C.c_double), ("enclosure", C.c_int32),
                ("split", C.c_int32)]


class gis_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("levels_done", C.c_int32), ("n_kept", C.c_int64), ("n_cells", C.c_int64),
                ("n_edges_total", C.c_int64), ("cells_built", C.c_int64), ("cells", C.POINTER(gis_cell)),
                ("cells_cap", C.c_int64)]


class gis_server_opts(C.Structure):
    _fields_ = [("max_active", C.c_int32), ("max_device_bytes", C.c_int64), ("lanes_per_pair", C.c_int32),
                ("timing", C.c_int32)]


_SERVER_STAT_FIELDS = [(k, C.c_int64) for k in ("submitted", "completed", "failed", "active", "queued", "steps",
                                                "cells_built", "cell_edges", "budget_bytes", "admitted_bytes",
                                                "oom_restarts", "peak_device_bytes")]


class gis_server_stats(C.Structure):
    _fields_ = _SERVER_STAT_FIELDS


# Names and signatures of every entry point of include/gis.h.
SIGNATURES = {
    "gis_default_options": (None, [C.POINTER(gis_options)]),
    "gis_create": (C.c_int32, [C.POINTER(C.c_void_p), C.POINTER(gis_dynamics), C.POINTER(gis_grid),
                               C.POINTER(gis_controls), C.POINTER(gis_options), C.c_void_p]),
    "gis_build_graph": (C.c_int32, [C.c_void_p]),
    "gis_prune": (C.c_int32, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int32)]),
    "gis_subdivide": (C.c_int32, [C.c_void_p, C.POINTER(C.c_int64)]),
    "gis_solve": (C.c_int32, [C.c_void_p, C.c_int32]),
    "gis_get_cells": (C.c_int32, [C.c_void_p, C.POINTER(gis_cell), C.c_int64, C.POINTER(C.c_int64)]),
    "gis_get_graph": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                  C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "gis_get_boxes": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64]),
    "gis_get_stats": (C.c_int32, [C.c_void_p, C.POINTER(gis_stats)]),
    "gis_last_error": (C.c_char_p, [C.c_void_p]),
    "gis_destroy": (None, [C.c_void_p]),
    "gis_batch_solve": (C.c_int32, [C.POINTER(gis_request), C.c_int32, C.POINTER(gis_result),
                                    C.POINTER(gis_options), C.c_void_p, C.POINTER(gis_stats)]),
    "gis_server_create": (C.c_int32, [C.POINTER(C.c_void_p), C.POINTER(gis_server_opts), C.c_int32]),
    "gis_server_submit": (C.c_int32, [C.c_void_p, C.POINTER(gis_request), C.POINTER(C.c_uint64)]),
    "gis_server_poll": (C.c_int32, [C.c_void_p, C.c_uint64, C.POINTER(gis_result), C.POINTER(C.c_int32), C.c_int32]),
    "gis_server_get_stats": (C.c_int32, [C.c_void_p, C.POINTER(gis_server_stats)]),
    "gis_server_destroy": (None, [C.c_void_p]),
    "gis_prune_graph_noalloc": (C.c_int32, [C.c_int64, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                            C.c_int32, C.c_void_p, C.POINTER(C.c_int64), C.c_void_p]),
    "gis_shard_create": (C.c_int32, [C.POINTER(C.c_void_p), C.c_int64, C.c_int64, C.c_int64, C.c_int32, C.c_void_p,
                                     C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "gis_shard_round": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int64)]),
    "gis_shard_kept": (C.c_int32, [C.c_void_p, C.c_void_p, C.POINTER(C.c_int64)]),
    "gis_shard_destroy": (None, [C.c_void_p]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libgis.so (built by paper_2202_06111_gb300.build); raise if missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"libgis.so not built ({path}); run paper_2202_06111_gb300.build.build()")
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc, ctx=None):
    if rc != OK:
        msg = load().gis_last_error(ctx)
        raise GisError(rc, msg.decode() if msg else "")


def current_stream() -> int:
    """The cudaStream_t of torch's current stream (0 = legacy default)."""
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return 0


def _dynamics(p: dict) -> gis_dynamics:
    d = gis_dynamics()
    d.dyn_id = DYN_IDS[p["dyn"]]
    d.n = p["n"]
    d.m = p.get("m", 1)
    d.substeps = p["substeps"]
    d.dt = p["dt"]
    for i, v in enumerate(p.get("params", [])):
        d.params[i] = v
    return d


def _grid(p: dict) -> gis_grid:
    g = gis_grid()
    for d in range(p["n"]):
        g.lo[d] = p["lo"][d]
        g.hi[d] = p["hi"][d]
        g.root_cells[d] = p["n0"][d]
    g.k_samples = p["k"]
    return g


def _controls(p: dict):
    u = np.ascontiguousarray(np.asarray(p["controls"], np.float64).reshape(-1, p.get("m", 1)))
    c = gis_controls()
    c.n_controls = u.shape[0]
    c.u = u.ctypes.data_as(C.POINTER(C.c_double))
    return c, u


def options(p: dict | None = None, **kw) -> gis_options:
    o = gis_options()
    load().gis_default_options(C.byref(o))
    if p is not None:
        o.rule = RULES[p.get("rule", "inner")]
        o.precision = PRECISIONS[p.get("precision", "fp32")]
        if "band" in p:
            o.band = p["band"]
        if "split_ring" in p:
            o.split_ring = int(p["split_ring"])
        o.enclosure = ENCLOSURES[p.get("enclosure", "samples")]
        o.split = SPLITS[p.get("split", "all")]
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Context:
    """One GIS problem on the GPU (gis_create ... gis_destroy)."""

    def __init__(self, prob: dict, stream: int | None = None, **opts):
        L = load()
        self.prob = prob
        self.n = prob["n"]
        self._dyn, self._grid = _dynamics(prob), _grid(prob)
        self._ctl, self._u = _controls(prob)
        self.n_u = self._u.shape[0]
        self._opt = options(prob, **opts)
        h = C.c_void_p()
        rc = L.gis_create(C.byref(h), C.byref(self._dyn), C.byref(self._grid), C.byref(self._ctl),
                          C.byref(self._opt), C.c_void_p(current_stream() if stream is None else stream))
        _check(rc)
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().gis_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def build_graph(self):
        _check(load().gis_build_graph(self._h), self._h)

    def prune(self):
        nk, nr = C.c_int64(), C.c_int32()
        _check(load().gis_prune(self._h, C.byref(nk), C.byref(nr)), self._h)
        return nk.value, nr.value

    def subdivide(self) -> int:
        ns = C.c_int64()
        _check(load().gis_subdivide(self._h, C.byref(ns)), self._h)
        return ns.value

    def solve(self, levels: int | None = None):
        _check(load().gis_solve(self._h, self.prob.get("levels", 0) if levels is None else levels), self._h)

    def cells(self):
        """(level[N], flags[N], idx[N, n]) of the live cells, in slot order:
        column views of one (N, 2 + MAXN) int32 array that the library fills
        (gis_cell rows; not zeroed first, nothing copied after)."""
        L = load()
        n = C.c_int64()
        _check(L.gis_get_cells(self._h, None, 0, C.byref(n)), self._h)
        a = np.empty((max(n.value, 1), 2 + MAXN), np.int32)
        _check(L.gis_get_cells(self._h, a.ctypes.data_as(C.POINTER(gis_cell)), n.value, C.byref(n)), self._h)
        a = a[:n.value]
        return a[:, 0], a[:, 1], a[:, 2:2 + self.n]

    def kept_cells(self):
        lv, fl, idx = self.cells()
        k = (fl & CELL_KEPT) != 0
        return lv[k], idx[k]

    def graph(self):
        """(off[P+1], tgt[E] as cell indices of cells(), flag[P])."""
        L = load()
        npairs, ne = C.c_int64(), C.c_int64()
        _check(L.gis_get_graph(self._h, None, None, None, 0, C.byref(npairs), C.byref(ne)), self._h)
        off = np.zeros(npairs.value + 1, np.int64)
        tgt = np.zeros(max(ne.value, 1), np.int32)
        flag = np.zeros(max(npairs.value, 1), np.uint8)
        _check(L.gis_get_graph(self._h, off.ctypes.data, tgt.ctypes.data, flag.ctypes.data, ne.value,
                               C.byref(npairs), C.byref(ne)), self._h)
        return off, tgt[:ne.value], flag[:npairs.value]

    def boxes(self):
        """(box32[P, 2n], box64[P, 2n], exact[P]) of the current pairs."""
        P = self.stats()["n_pairs"]
        b32 = np.zeros((max(P, 1), 2 * self.n), np.float32)
        b64 = np.zeros((max(P, 1), 2 * self.n), np.float64)
        ex = np.zeros(max(P, 1), np.uint8)
        _check(load().gis_get_boxes(self._h, b32.ctypes.data, b64.ctypes.data, ex.ctypes.data, P), self._h)
        return b32[:P], b64[:P], ex[:P]

    def stats(self) -> dict:
        s = gis_stats()
        _check(load().gis_get_stats(self._h, C.byref(s)), self._h)
        return {k: getattr(s, k) for k, _ in _STAT_FIELDS}


def batch_solve(problems: list[dict], stream: int | None = None, want_cells: bool = True, **opts):
    """gis_batch_solve over problem dicts; returns (results, stats) with each
    result a dict (status, n_kept, n_cells, n_edges_total, cells_built, levels_done,
    kept = (level, idx) if want_cells). A problem's kept-cell buffer holds
    `cells_cap` cells (default 2 x root cells x (1 + levels)); beyond it the
    list is cut while n_kept stays exact."""
    L = load()
    n = len(problems)
    reqs = (gis_request * max(n, 1))()
    res = (gis_result * max(n, 1))()
    keep = []
    cell_bufs = []
    for i, p in enumerate(problems):
        r = reqs[i]
        r.dyn = _dynamics(p)
        r.grid = _grid(p)
        c, u = _controls(p)
        keep.append(u)
        r.controls = c
        r.levels = p.get("levels", 0)
        r.rule = RULES[p.get("rule", "inner")]
        r.precision = PRECISIONS[p.get("precision", "fp32")]
        r.band = p.get("band", 0.0)
        r.enclosure = ENCLOSURES[p.get("enclosure", "samples")]
        r.split = SPLITS[p.get("split", "all")]
        if want_cells:
            cap = p.get("cells_cap", 2 * int(np.prod(p["n0"])) * (1 + r.levels))
            buf = (gis_cell * cap)()
            cell_bufs.append(buf)
            res[i].cells = C.cast(buf, C.POINTER(gis_cell))
            res[i].cells_cap = cap
        else:
            cell_bufs.append(None)
    o = options(None, **opts)
    st = gis_stats()
    rc = L.gis_batch_solve(reqs, n, res, C.byref(o), C.c_void_p(current_stream() if stream is None else stream),
                           C.byref(st))
    _check(rc)
    out = []
    for i, p in enumerate(problems):
        r = res[i]
        d = {"status": r.status, "n_kept": r.n_kept, "n_cells": r.n_cells, "n_edges_total": r.n_edges_total,
             "cells_built": r.cells_built, "levels_done": r.levels_done}
        if want_cells:
            a = np.frombuffer(cell_bufs[i], dtype=np.int32).reshape(-1, 2 + MAXN)[:r.n_kept]
            d["kept"] = (a[:, 0].copy(), a[:, 2:2 + p["n"]].copy())
        out.append(d)
    return out, {k: getattr(st, k) for k, _ in _STAT_FIELDS}


def _request(p: dict, keep: list) -> gis_request:
    r = gis_request()
    r.dyn = _dynamics(p)
    r.grid = _grid(p)
    c, u = _controls(p)
    keep.append(u)
    r.controls = c
    r.levels = p.get("levels", 0)
    r.rule = RULES[p.get("rule", "inner")]
    r.precision = PRECISIONS[p.get("precision", "fp32")]
    r.band = p.get("band", 0.0)
    r.enclosure = ENCLOSURES[p.get("enclosure", "samples")]
    r.split = SPLITS[p.get("split", "all")]
    return r


class Server:
    """Continuous-batching server (gis_server_*): submit problems at any time,
    poll or wait for their kept cells."""

    def __init__(self, device: int = 0, max_active: int = 0, max_device_bytes: int = 0, lanes_per_pair: int = 0):
        L = load()
        o = gis_server_opts(max_active, max_device_bytes, lanes_per_pair, 0)
        h = C.c_void_p()
        _check(L.gis_server_create(C.byref(h), C.byref(o), device))
        self._h = h
        self._meta = {}

    def submit(self, prob: dict) -> int:
        keep = []
        r = _request(prob, keep)
        t = C.c_uint64()
        _check(load().gis_server_submit(self._h, C.byref(r), C.byref(t)))
        self._meta[t.value] = prob
        return t.value

    def poll(self, ticket: int, wait: bool = False, want_cells: bool = True):
        """None while running; else a result dict (as batch_solve's)."""
        prob = self._meta[ticket]
        res = gis_result()
        buf = None
        if want_cells:
            cap = prob.get("cells_cap", 2 * int(np.prod(prob["n0"])) * (1 + prob.get("levels", 0)))
            buf = (gis_cell * cap)()
            res.cells = C.cast(buf, C.POINTER(gis_cell))
            res.cells_cap = cap
        done = C.c_int32()
        rc = load().gis_server_poll(self._h, ticket, C.byref(res), C.byref(done), 1 if wait else 0)
        if rc == EBOUNDS and want_cells:          # buffer too small: size it from the result
            cap = res.n_kept
            buf = (gis_cell * max(cap, 1))()
            res.cells = C.cast(buf, C.POINTER(gis_cell))
            res.cells_cap = cap
            rc = load().gis_server_poll(self._h, ticket, C.byref(res), C.byref(done), 1)
        _check(rc)
        if not done.value:
            return None
        del self._meta[ticket]
        d = {"status": res.status, "n_kept": res.n_kept, "n_cells": res.n_cells, "n_edges_total": res.n_edges_total,
             "cells_built": res.cells_built, "levels_done": res.levels_done}
        if want_cells:
            a = np.frombuffer(buf, dtype=np.int32).reshape(-1, 2 + MAXN)[:min(res.n_kept, res.cells_cap)]
            d["kept"] = (a[:, 0].copy(), a[:, 2:2 + prob["n"]].copy())
        return d

    def stats(self) -> dict:
        s = gis_server_stats()
        _check(load().gis_server_get_stats(self._h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in _SERVER_STAT_FIELDS}

    def close(self):
        if getattr(self, "_h", None):
            load().gis_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
