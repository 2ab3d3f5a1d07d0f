"""The C-ABI library builds, loads and exports every entry point of include/rt.h;
argument validation answers without touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_0903_1949_gb300 import build as B
from paper_0903_1949_gb300 import inputs as I
from paper_0903_1949_gb300 import rt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return rt.load()


def declared():
    src = open(os.path.join(ROOT, "include", "rt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rt_[A-Za-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), n


def test_binding_names_match_abi(lib):
    for n in declared():
        assert hasattr(rt, n), n


def _desc(**over):
    e = I.sph_edges(4, 3, 5)
    dirs, w = I.angle_set(2, 2)
    kw = dict(coord=I.SPHERICAL, edges=e, dirs=dirs, weights=w)
    kw.update(over)
    return kw


@pytest.mark.parametrize("bad", [
    dict(coord=7),
    dict(edges=[np.array([1.0, 0.5, 2.0]), I.sph_edges(4, 3, 5)[1], I.sph_edges(4, 3, 5)[2]]),
    dict(edges=[np.array([0.0, 1.0, 2.0]), I.sph_edges(4, 3, 5)[1], I.sph_edges(4, 3, 5)[2]]),
    dict(edges=[I.sph_edges(4, 3, 5)[0], np.linspace(0.0, 3.0, 4), I.sph_edges(4, 3, 5)[2]]),
    dict(edges=[I.sph_edges(4, 3, 5)[0], I.sph_edges(4, 3, 5)[1], np.linspace(0.0, 6.0, 6)]),
    dict(weights=np.full(4, 0.3)),
    dict(dirs=np.ones((4, 3))),
    dict(inner_bc=5),
    dict(precision=3),
    dict(angle_block=300),
    dict(I_outer=-1.0),
])
def test_invalid_descriptions_are_rejected(lib, bad):
    kw = _desc(**bad)
    with pytest.raises(rt.RtError) as ei:
        rt.rt_grid_create(**kw)
    assert ei.value.code == rt.RT_EINVAL
    assert len(rt.rt_last_error()) > 0


def test_too_many_voxels_rejected(lib):
    """Voxel ids live in 28 bits of the segment word: 1024 x 512 x 1024 voxels (2^29) is refused
    before any device work."""
    e = I.sph_edges(1024, 512, 1024)
    with pytest.raises(rt.RtError) as ei:
        rt.rt_grid_create(**_desc(edges=e))
    assert ei.value.code == rt.RT_EINVAL
    assert "too many voxels" in str(ei.value)


def test_zero_angles_rejected(lib):
    with pytest.raises(rt.RtError) as ei:
        rt.rt_grid_create(**_desc(dirs=np.zeros((0, 3)), weights=np.zeros(0)))
    assert ei.value.code == rt.RT_EINVAL


def test_null_handles_rejected(lib):
    assert lib.rt_formal_solution(None) == rt.RT_EINVAL
    assert lib.rt_ali_step(None, None) == rt.RT_EINVAL
    assert lib.rt_grid_destroy(None) == rt.RT_OK
    out = np.zeros(4)
    assert lib.rt_get_J(None, ctypes.c_void_p(out.ctypes.data), rt.RT_HOST) == rt.RT_EINVAL
    p = ctypes.c_void_p(out.ctypes.data)
    assert lib.rt_adjoint(None, None, None, None, 1e-8, 10, p, p, p, rt.RT_HOST, None) == rt.RT_EINVAL
    h = ctypes.c_void_p()
    assert lib.rt_line_create(ctypes.byref(h), None, 4, p, p, rt.RT_LSTAR_DIAG, 0, None) == rt.RT_EINVAL
    assert lib.rt_line_set(None, p, p, p, p, rt.RT_HOST) == rt.RT_EINVAL
    assert lib.rt_line_step(None, None) == rt.RT_EINVAL
    assert lib.rt_line_solve(None, 1e-6, 10, None) == rt.RT_EINVAL
    assert lib.rt_line_get(None, 0, p, rt.RT_HOST) == rt.RT_EINVAL


def test_library_wide_knob_takes_a_null_grid(lib):
    assert lib.rt_tune(None, rt.RT_TUNE_GEOM_PREDICT, 2) == rt.RT_EINVAL
    assert lib.rt_tune(None, rt.RT_TUNE_GEOM_PREDICT, 1) == rt.RT_OK
    assert lib.rt_tune(None, rt.RT_TUNE_GEOM_PREDICT, 0) == rt.RT_OK
    assert lib.rt_tune(None, rt.RT_TUNE_GRAPH, 1) == rt.RT_EINVAL  # the other knobs need a grid


def test_struct_layout_matches_header(lib):
    # rt_grid_desc / rt_info sizes as laid out by the C compiler for x86-64 and aarch64
    assert ctypes.sizeof(rt.rt_grid_desc) == 112
    assert ctypes.sizeof(rt.rt_info) == 80
    assert ctypes.sizeof(rt.rt_timing) == 88


def test_struct_offsets_match_the_c_compiler(tmp_path):
    """Every field offset and struct size of the binding's ctypes structs equals
    what gcc lays out from include/rt.h on this machine."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no gcc")
    structs = [rt.rt_grid_desc, rt.rt_info, rt.rt_timing]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "rt.h"', "int main(void) {"]
    for st in structs:
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (st.__name__, st.__name__))
        for name, _ in st._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (st.__name__, name, st.__name__, name))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run(["gcc", "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                  check=True).stdout.splitlines())
    for st in structs:
        assert int(got[st.__name__]) == ctypes.sizeof(st), st.__name__
        for name, _ in st._fields_:
            assert int(got["%s.%s" % (st.__name__, name)]) == getattr(st, name).offset, (st.__name__, name)
