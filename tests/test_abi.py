"""The C ABI library loads without a GPU and exports exactly what include/gis.h
declares; the ctypes structs match the C layout (checked by compiling a probe
of the header with gcc)."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2202_06111_gb300 import build as B
from paper_2202_06111_gb300 import gis

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gis.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+char\s*\*|gis_status|void)\s*\**\s*(gis_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return gis.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(gis.SIGNATURES) == names


def test_struct_layouts_match_header(tmp_path):
    probe = tmp_path / "probe.c"
    structs = ["gis_dynamics", "gis_grid", "gis_controls", "gis_options", "gis_cell", "gis_stats",
               "gis_request", "gis_result"]
    probe.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "gis.h"\nint main(void){\n' +
                     "".join(f'printf("{s} %zu\\n", sizeof({s}));\n' for s in structs) +
                     'printf("off_band %zu\\n", offsetof(gis_options, band));\n'
                     'printf("off_cells %zu\\n", offsetof(gis_result, cells));\n'
                     'printf("off_prune_bytes %zu\\n", offsetof(gis_stats, prune_bytes));\nreturn 0;}\n')
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.dirname(HEADER), str(probe), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    for s in structs:
        assert int(out[s]) == C.sizeof(getattr(gis, s)), s
    assert int(out["off_band"]) == gis.gis_options.band.offset
    assert int(out["off_cells"]) == gis.gis_result.cells.offset
    assert int(out["off_prune_bytes"]) == gis.gis_stats.prune_bytes.offset


def test_default_options(lib):
    o = gis.options()
    assert o.rule == 0 and o.precision == 1 and o.band == 0.0 and o.lanes_per_pair == 0
    assert o.fixed_shapes == 0 and o.split_ring == 0 and o.enclosure_store == 0 and o.max_device_bytes == 0
    p = gis.options({"rule": "outer", "split_ring": 3}, fixed_shapes=1)
    assert p.rule == 1 and p.split_ring == 3 and p.fixed_shapes == 1


def test_null_arguments_rejected_without_touching_a_gpu(lib):
    h = C.c_void_p()
    assert lib.gis_create(C.byref(h), None, None, None, None, None) == gis.EINVAL
    assert lib.gis_build_graph(None) == gis.EINVAL
    assert lib.gis_prune(None, None, None) == gis.EINVAL
    assert lib.gis_solve(None, 0) == gis.EINVAL
    lib.gis_destroy(None)
    assert isinstance(lib.gis_last_error(None), bytes)
