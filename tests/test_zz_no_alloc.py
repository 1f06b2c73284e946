"""canvox_render_noalloc: the entry point for callers that cannot allocate device memory.

It renders from caller-owned device buffers and keeps its working memory in a
fixed device array, so it must give the same image as canvox_render, call
after call (the array keeps the previous call's contents), and match the FP64
oracle like every other render. This file is collected last so that a failure
here does not hide the other tests.
"""
import numpy as np
import pytest

import oracle
import paper_1704_02724_gb300 as cx
from paper_1704_02724_gb300 import canvox
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def _views():
    cams = list(synth.config_cameras(0, res_scale=0.5))
    off = synth.total_pixels(cams)
    cams.append(synth.look_at_camera([0.1, 0.05, -0.2], [0.3, 0.1, 0.4], [0, 1, 0], 1.0, 37, 23, off,
                                     (0.1, 0.2, 0.3, 1.0)))
    return synth.cameras_array(cams)


def test_noalloc_matches_render_on_two_calls():
    from paper_1704_02724_gb300 import _build
    _build.build()
    cv = synth.build_config(0)
    cams = _views()
    n = synth.total_pixels(cams)
    # reference: the allocating entry point
    cx.upload_octree(cv.nodes, cv.leaves, cv.depth, cv.extent)
    ref = torch.full((n, 4), float("nan"), device="cuda")
    cx.render(cams, ref)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    ref_oracle = oracle.render(cv, cams)
    # caller-owned device copies of the pools
    nodes = torch.from_numpy(np.ascontiguousarray(cv.nodes)).cuda()
    leaves = torch.from_numpy(np.ascontiguousarray(cv.leaves).view(np.int16)).cuda()
    for _ in range(2):
        out = torch.full((n, 4), float("nan"), device="cuda")
        cx.render_noalloc(nodes, cv.n_records, leaves, cv.n_leaves, cv.depth, cv.extent, cams, out)
        torch.cuda.synchronize()
        img = out.cpu().numpy()
        assert np.all(np.isfinite(img))
        assert float(np.max(np.abs(img.astype(np.float64) - ref))) <= TOL
        assert float(np.max(np.abs(img.astype(np.float64) - ref_oracle))) <= TOL


def test_noalloc_rejects_too_many_views():
    cv = synth.build_config(0)
    cams = synth.cameras_array([synth.config_cameras(0, res_scale=0.05)[0]] * 65)
    nodes = torch.from_numpy(np.ascontiguousarray(cv.nodes)).cuda()
    leaves = torch.from_numpy(np.ascontiguousarray(cv.leaves).view(np.int16)).cuda()
    out = torch.zeros((synth.total_pixels(cams), 4), device="cuda")
    with pytest.raises(cx.CanvoxError) as e:
        cx.render_noalloc(nodes, cv.n_records, leaves, cv.n_leaves, cv.depth, cv.extent, cams, out)
    assert e.value.code == canvox.ERR_INVALID_ARG and "64 views" in str(e.value)
    with pytest.raises(cx.CanvoxError) as e:   # pool sizes beyond int32 indices are refused before any launch
        cx.render_noalloc(nodes, 2 ** 31, leaves, cv.n_leaves, cv.depth, cv.extent, cams[:1], out)
    assert e.value.code == canvox.ERR_INVALID_ARG
