"""The C ABI boundary on CPU: the library loads, exports every declared entry
point, its structs match the Python mirrors, and host-side validation rejects
bad input before touching a GPU."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import paper_1704_02724_gb300 as cx
from paper_1704_02724_gb300 import _build, canvox
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "canvox.h")


@pytest.fixture(scope="module")
def L():
    _build.build()
    return cx.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(canvox_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(L, n), n


def test_struct_layouts_match_header(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "canvox.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu\\n\", sizeof(canvox_camera), sizeof(canvox_render_opts),"
        " sizeof(canvox_stats), offsetof(canvox_camera, background), offsetof(canvox_render_opts, step_count),"
        " offsetof(canvox_camera, out_offset_px)); return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    cam, opts, stats, bg_off, sc_off, off_off = map(int, subprocess.run([str(exe)], capture_output=True, text=True).stdout.split())
    assert cam == synth.CAM_DTYPE.itemsize == canvox.CAMERA_BYTES
    assert bg_off == synth.CAM_DTYPE.fields["background"][1]
    assert off_off == synth.CAM_DTYPE.fields["out_offset_px"][1]
    assert opts == ctypes.sizeof(canvox.Opts) and sc_off == canvox.Opts.step_count.offset
    assert stats == ctypes.sizeof(canvox.Stats)


def test_host_paths_without_gpu(L):
    d = cx.default_opts()
    assert d["precision"] == cx.PREC_MIXED and d["frame_levels"] == 20 and d["refill"] == 0
    s = cx.get_stats()
    assert s["rays"] == 0
    cams = synth.config_cameras(0)
    with pytest.raises(cx.CanvoxError) as e:
        cx.render(cams, 0, stream=0)                  # null output
    assert e.value.code == canvox.ERR_INVALID_ARG
    with pytest.raises(cx.CanvoxError) as e:
        cx.render(cams, 1 << 40, stream=0)            # never dereferenced: nothing uploaded
    assert e.value.code == canvox.ERR_NOT_UPLOADED
    with pytest.raises(cx.CanvoxError) as e:
        cx.octree_hash()
    assert e.value.code == canvox.ERR_NOT_UPLOADED
    with pytest.raises(cx.CanvoxError) as e:
        cx.update_leaves(0, np.zeros((1, 4), np.uint16))
    assert e.value.code == canvox.ERR_NOT_UPLOADED
    with pytest.raises(cx.CanvoxError) as e:
        cx.paint_append(np.zeros((1, 3)), [0.1], [[1, 1, 1, 1]])
    assert e.value.code == canvox.ERR_NOT_UPLOADED


def _expect(code, nodes, leaves, depth=4, extent=1.0):
    with pytest.raises(cx.CanvoxError) as e:
        cx.upload_octree(nodes, leaves, depth, extent)
    assert e.value.code == code, str(e.value)


def test_upload_validation_rejects_bad_pools(L):
    half = np.float16(np.array([0.5, 0.5, 0.5, 2.0])).view(np.uint16)
    ok_nodes = np.array([[1, 0, -1, 0, 0, 0, 0, 0], [0, -2, 0, 0, 0, 0, 0, 0]], np.int32)
    ok_leaves = np.array([half, half], np.uint16)
    # argument errors
    _expect(canvox.ERR_INVALID_ARG, ok_nodes, ok_leaves, depth=0)
    _expect(canvox.ERR_INVALID_ARG, ok_nodes, ok_leaves, depth=31)
    _expect(canvox.ERR_INVALID_ARG, ok_nodes, ok_leaves, extent=-1.0)
    _expect(canvox.ERR_INVALID_ARG, ok_nodes, ok_leaves, extent=1.0 + 2.0 ** -30)   # > 23 significant bits
    # structure errors
    bad = ok_nodes.copy(); bad[0, 0] = 2
    _expect(canvox.ERR_BAD_TREE, bad, ok_leaves)                                 # child out of range
    bad = ok_nodes.copy(); bad[1, 0] = 1
    _expect(canvox.ERR_BAD_TREE, bad, ok_leaves)                                 # cycle / not breadth-first
    bad = ok_nodes.copy(); bad[0, 2], bad[1, 1] = -2, -1
    _expect(canvox.ERR_BAD_TREE, bad, ok_leaves)                                 # leaves out of order
    _expect(canvox.ERR_BAD_TREE, ok_nodes, ok_leaves[:1])                        # leaf index out of range
    _expect(canvox.ERR_BAD_TREE, ok_nodes, ok_leaves, depth=1)                   # record deeper than depth - 1
    nan = ok_leaves.copy(); nan[1, 3] = 0x7E00
    _expect(canvox.ERR_BAD_TREE, ok_nodes, nan)                                  # NaN extinction
    neg = ok_leaves.copy(); neg[0, 3] = np.float16(-1.0).view(np.uint16)
    _expect(canvox.ERR_BAD_TREE, ok_nodes, neg)                                  # negative extinction
    extra = np.vstack([ok_nodes, np.zeros((1, 8), np.int32)])
    _expect(canvox.ERR_BAD_TREE, extra, ok_leaves)                               # unreachable record
