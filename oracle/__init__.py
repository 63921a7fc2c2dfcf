"""FP64 CPU oracle of the GIS hot path -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline / reference leg
of ``bench.py`` may import this package. The CUDA library never calls it and it
shares no code with it: ``gis_oracle.c`` is a plain, slow FP64 restatement of
the method (cell covering Sec. 2.1, symbolic image Def. 1, pruning fixed point
Sec. 2.3 / Prop. 1, boundary rule Sec. 3.1.1 / Alg. 1, subdivision Sec. 3.1),
compiled without FMA contraction.

Problems are plain dicts (see ``paper_2202_06111_gb300.workloads``):
``dyn`` (name), ``n``, ``m``, ``params``, ``dt``, ``substeps``, ``lo``, ``hi``,
``n0``, ``k``, ``controls`` (n_u x m), ``rule`` ("inner" | "outer" | "scc": the
largest strongly connected component and its ancestors, Def. 3), optionally
``enclosure`` ("samples": the bounding box of the sample lattice, default;
"interval": an interval enclosure of the whole cell's image), ``split`` ("all":
2^n children, default; "cycled": 2 children halving one dimension, cycled), optionally
``split_ring`` (cells split besides the boundary cells: those within this many
rings of them, -1 every kept cell; default 0).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gis_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

DYN_IDS = {"linmap": 0, "vdp": 1, "cstr_dl": 2, "cartpole": 3, "cstr_paper": 4}
RULES = {"inner": 0, "outer": 1, "scc": 2}
F_INX, F_TOUCH_DEAD, F_NONFINITE = 1, 2, 4
DEAD, ALIVE, SPLIT = 0, 1, 2
MAXN = 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no contraction, OpenMP if present)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
            "-shared", "-o", _LIB, _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    return _LIB


class _Problem(C.Structure):
    _fields_ = [("dyn", C.c_int32), ("n", C.c_int32), ("m", C.c_int32), ("substeps", C.c_int32),
                ("dt", C.c_double), ("p", C.c_double * 32),
                ("lo", C.c_double * MAXN), ("hi", C.c_double * MAXN),
                ("n0", C.c_int32 * MAXN), ("k", C.c_int32), ("rule", C.c_int32), ("enclosure", C.c_int32),
                ("split", C.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        vp, i32, i64, dp = C.c_void_p, C.c_int32, C.c_int64, C.POINTER(C.c_double)
        L.orc_create.restype = vp
        L.orc_create.argtypes = [C.POINTER(_Problem), dp, i32]
        L.orc_destroy.argtypes = [vp]
        for name in ("orc_build_graph",):
            getattr(L, name).argtypes = [vp]
        L.orc_prune.argtypes = [vp, C.POINTER(i64)]
        L.orc_subdivide.argtypes = [vp, C.POINTER(i64)]
        L.orc_classify.argtypes = [vp, vp, C.POINTER(i64)]
        L.orc_solve.argtypes = [vp, i32]
        L.orc_set_kept.argtypes = [vp, vp]
        L.orc_set_ring.argtypes = [vp, i32]
        for name in ("orc_num_live", "orc_num_edges", "orc_num_nodes"):
            getattr(L, name).restype = i64
            getattr(L, name).argtypes = [vp]
        L.orc_max_level.restype = i32
        L.orc_max_level.argtypes = [vp]
        L.orc_get_live.argtypes = [vp, vp, vp]
        L.orc_get_graph.argtypes = [vp, vp, vp, vp, vp]
        L.orc_get_kept.argtypes = [vp, vp]
        L.orc_get_nodes.argtypes = [vp, vp, vp, vp, vp]
        L.orc_rhs.argtypes = [C.POINTER(_Problem), vp, vp, vp]
        L.orc_step.argtypes = [C.POINTER(_Problem), vp, vp, vp]
        L.orc_cell_samples.argtypes = [C.POINTER(_Problem), i32, vp, vp]
        L.orc_pair_bbox.argtypes = [C.POINTER(_Problem), i32, vp, vp, vp, vp]
        L.orc_range.argtypes = [C.POINTER(_Problem), i32, i32, C.c_double, C.c_double, vp]
        L.orc_prune_graph.argtypes = [i64, i32, vp, vp, vp, i32, vp, C.POINTER(i64)]
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_build_slice.argtypes = [vp, i64, i64, C.POINTER(i64)]
        L.orc_own_exp.restype = C.c_double
        L.orc_own_exp.argtypes = [C.c_double]
        L.orc_own_sincos.argtypes = [C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        _lib = L
    return _lib


def set_threads(t: int = 0) -> int:
    """Threads for the per-pair loop of graph construction (0: all cores)."""
    return lib().orc_set_threads(t)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _struct(prob: dict) -> _Problem:
    s = _Problem()
    s.dyn = DYN_IDS[prob["dyn"]]
    s.n = prob["n"]
    s.m = prob.get("m", 1)
    s.substeps = prob["substeps"]
    s.dt = prob["dt"]
    for i, v in enumerate(prob.get("params", [])):
        s.p[i] = v
    for d in range(prob["n"]):
        s.lo[d] = prob["lo"][d]
        s.hi[d] = prob["hi"][d]
        s.n0[d] = prob["n0"][d]
    s.k = prob["k"]
    s.rule = RULES[prob.get("rule", "inner")]
    s.enclosure = {"samples": 0, "interval": 1}[prob.get("enclosure", "samples")]
    s.split = {"all": 0, "cycled": 1}[prob.get("split", "all")]
    return s


def _check(rc):
    if rc != 0:
        raise RuntimeError(f"oracle error {rc}")


def rhs(prob, x, u):
    x = np.ascontiguousarray(x, np.float64)
    u = np.ascontiguousarray(u, np.float64)
    out = np.zeros(MAXN)
    _check(lib().orc_rhs(C.byref(_struct(prob)), _ptr(x), _ptr(u), _ptr(out)))
    return out[:prob["n"]]


def step(prob, x, u):
    x = np.ascontiguousarray(x, np.float64)
    u = np.ascontiguousarray(u, np.float64)
    out = np.zeros(MAXN)
    _check(lib().orc_step(C.byref(_struct(prob)), _ptr(x), _ptr(u), _ptr(out)))
    return out[:prob["n"]]


def cell_samples(prob, level, idx):
    n, k = prob["n"], prob["k"]
    idx = np.zeros(MAXN, np.int32) + np.pad(np.asarray(idx, np.int32), (0, MAXN - n))
    out = np.zeros((k ** n, n))
    _check(lib().orc_cell_samples(C.byref(_struct(prob)), level, _ptr(idx), _ptr(out)))
    return out


def pair_bbox(prob, level, idx, u):
    """(ymin, ymax, nonfinite) of one (cell, control) pair."""
    n = prob["n"]
    idx = np.pad(np.asarray(idx, np.int32), (0, MAXN - n))
    u = np.ascontiguousarray(u, np.float64)
    lo, hi = np.zeros(MAXN), np.zeros(MAXN)
    nf = lib().orc_pair_bbox(C.byref(_struct(prob)), level, _ptr(idx), _ptr(u), _ptr(lo), _ptr(hi))
    return lo[:n], hi[:n], bool(nf)


def own_exp(x: float) -> float:
    """The interval mode's own e^x (range reduction + Taylor)."""
    return lib().orc_own_exp(float(x))


def own_sincos(x: float):
    """The interval mode's own (sin x, cos x); None beyond |x| = 65536."""
    s, c = C.c_double(), C.c_double()
    ok = lib().orc_own_sincos(float(x), C.byref(s), C.byref(c))
    return (s.value, c.value) if ok else None


def level_range(prob, level, d, ymin, ymax):
    out = np.zeros(2, np.int64)
    _check(lib().orc_range(C.byref(_struct(prob)), level, d, float(ymin), float(ymax), _ptr(out)))
    return int(out[0]), int(out[1])


def prune_graph(n_cells, n_u, off, tgt, flag, rule="inner"):
    """Greatest fixed point of the pruning rule on an explicit graph."""
    off = np.ascontiguousarray(off, np.int64)
    tgt = np.ascontiguousarray(tgt, np.int32)
    flag = np.ascontiguousarray(flag, np.uint8)
    kept = np.zeros(max(n_cells, 1), np.uint8)
    nk = C.c_int64(0)
    _check(lib().orc_prune_graph(n_cells, n_u, _ptr(off), _ptr(tgt), _ptr(flag), RULES[rule],
                                 _ptr(kept), C.byref(nk)))
    return kept[:n_cells].astype(bool)


class Solver:
    """The GIS loop of Sec. 2 / Sec. 3 on one problem, in plain FP64."""

    def __init__(self, prob: dict):
        self.prob = prob
        self.n = prob["n"]
        ctrl = np.ascontiguousarray(np.asarray(prob["controls"], np.float64).reshape(-1, prob.get("m", 1)))
        self.n_u = ctrl.shape[0]
        self._s = _struct(prob)
        self._h = lib().orc_create(C.byref(self._s), ctrl.ctypes.data_as(C.POINTER(C.c_double)), self.n_u)
        if not self._h:
            raise ValueError("oracle: invalid problem")
        ring = int(prob.get("split_ring", 0))
        if ring:
            _check(lib().orc_set_ring(self._h, ring))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_destroy(h)
            self._h = None

    def build_graph(self):
        _check(lib().orc_build_graph(self._h))

    def build_slice(self, first: int, count: int) -> int:
        """Graph construction of live cells [first, first + count) of the
        current covering, discarded afterwards (a bounded timing sample);
        returns its edge count. The solver keeps no graph."""
        ne = C.c_int64(0)
        _check(lib().orc_build_slice(self._h, first, count, C.byref(ne)))
        return ne.value

    def prune(self) -> int:
        nk = C.c_int64(0)
        _check(lib().orc_prune(self._h, C.byref(nk)))
        return nk.value

    def classify(self):
        nl = self.num_live()
        bnd = np.zeros(max(nl, 1), np.uint8)
        nb = C.c_int64(0)
        _check(lib().orc_classify(self._h, _ptr(bnd), C.byref(nb)))
        return bnd[:nl].astype(bool)

    def subdivide(self) -> int:
        ns = C.c_int64(0)
        _check(lib().orc_subdivide(self._h, C.byref(ns)))
        return ns.value

    def solve(self, levels: int):
        _check(lib().orc_solve(self._h, levels))

    def set_kept(self, kept):
        k = np.ascontiguousarray(kept, np.uint8)
        _check(lib().orc_set_kept(self._h, _ptr(k)))

    def num_live(self) -> int:
        return lib().orc_num_live(self._h)

    def num_edges(self) -> int:
        return lib().orc_num_edges(self._h)

    def max_level(self) -> int:
        return lib().orc_max_level(self._h)

    def live(self):
        """(level[N], idx[N, n]) of the live cells in canonical order."""
        nl = self.num_live()
        lv = np.zeros(max(nl, 1), np.int32)
        idx = np.zeros((max(nl, 1), MAXN), np.int32)
        _check(lib().orc_get_live(self._h, _ptr(lv), _ptr(idx)))
        return lv[:nl], idx[:nl, :self.n]

    def graph(self):
        """(off, tgt, flag, bbox[P, 2n]) of the current graph, canonical slots."""
        nl, ne = self.num_live(), self.num_edges()
        P = nl * self.n_u
        off = np.zeros(P + 1, np.int64)
        tgt = np.zeros(max(ne, 1), np.int32)
        flag = np.zeros(max(P, 1), np.uint8)
        bbox = np.zeros((max(P, 1), 2 * self.n))
        _check(lib().orc_get_graph(self._h, _ptr(off), _ptr(tgt), _ptr(flag), _ptr(bbox)))
        return off, tgt[:ne], flag[:P], bbox[:P]

    def kept(self):
        nl = self.num_live()
        k = np.zeros(max(nl, 1), np.uint8)
        _check(lib().orc_get_kept(self._h, _ptr(k)))
        return k[:nl].astype(bool)

    def kept_cells(self):
        """(level[K], idx[K, n]) of the kept cells, canonical order."""
        lv, idx = self.live()
        k = self.kept()
        return lv[k], idx[k]

    def nodes(self):
        nn = lib().orc_num_nodes(self._h)
        lv = np.zeros(nn, np.int32)
        st = np.zeros(nn, np.int32)
        idx = np.zeros((nn, MAXN), np.int32)
        ch = np.zeros(nn, np.int64)
        _check(lib().orc_get_nodes(self._h, _ptr(lv), _ptr(st), _ptr(idx), _ptr(ch)))
        return lv, st, idx[:, :self.n], ch


def solve(prob: dict, levels: int | None = None) -> Solver:
    s = Solver(prob)
    s.solve(prob.get("levels", 0) if levels is None else levels)
    return s
