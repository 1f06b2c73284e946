"""The paper's single-precision walks on a GPU (Sec. 6.2-6.3; Fig. rayAngleError and the
canvas-vs-cell coordinate comparison): the cell-local FP32 walk keeps the ray-angle error
small at any depth, the same walk in FP32 canvas coordinates drifts, the cell-local walk
in binary16 stays within the same bound with eps = 2^-10, and the library's
mixed-precision path meets the 1e-5 bar where none of them does."""
import math

import numpy as np
import pytest

import oracle
import paper_1704_02724_gb300 as cx
import synth
from gpu_util import TOL, config_canvas, max_err, render
from test_parity_gpu import _embedded_scene

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = 2.0 ** -23   # the paper's machine epsilon for FP32
EPS16 = 2.0 ** -10  # binary16 (the half-precision remark of Sec. 6.3)


def _angles(cv, cams, key, prec):
    n = synth.total_pixels(cams)
    ang = torch.full((n,), float("nan"), device="cuda")
    img, st = render(cv, cams, key=key, precision=prec, angle_deg=ang)
    return img, ang.cpu().numpy().astype(np.float64)


def test_cell_local_walk_shallow_canvas():
    cv = config_canvas(0)
    cams = synth.config_cameras(0)
    ref = oracle.render(cv, cams)
    img, ang = _angles(cv, cams, "c0", cx.PREC_CELL32)
    assert np.all(np.isfinite(img)) and np.all(np.isfinite(ang))
    assert max_err(img, ref) <= 1e-3
    # every ray starts on the cube, in a cell of side at most 1/2, at least 1.5 units from the eye
    e0 = math.sqrt(3) * 2.0 ** -25 * 2.0 ** -1
    bound = math.degrees(math.asin(math.sqrt(2) * (e0 / 1.5 + 7.5 * EPS)))
    assert np.max(ang) <= bound
    # the same walk in binary16: the same bound with eps = 2^-10 (and e0 of a binary16 start point)
    img16, ang16 = _angles(cv, cams, "c0", cx.PREC_CELL16)
    assert np.all(np.isfinite(img16)) and np.all(np.isfinite(ang16))
    e0_16 = math.sqrt(3) * 2.0 ** -12 * 2.0 ** -1
    bound16 = math.degrees(math.asin(math.sqrt(2) * (e0_16 / 1.5 + 7.5 * EPS16)))
    assert np.max(ang16) <= bound16
    assert np.max(ang16) > 10 * np.max(ang)
    assert np.median(np.abs(img16 - ref).max(axis=1)) <= 0.05  # wrong cells only along silhouettes


@pytest.mark.parametrize("level", [23, 26])
def test_angle_error_cell_vs_canvas_coordinates(level):
    cv, lo, s = _embedded_scene(level)
    centre = lo + 0.5 * s
    cams = synth.cameras_array([
        synth.look_at_camera(centre + np.array([1.3, 0.7, -1.9]) * s, centre, [0, 1, 0], 0.5, 48, 40, 0)])
    ref = oracle.render(cv, cams)
    mixed, _ = render(cv, cams, key=("deep", level))
    cell, a_cell = _angles(cv, cams, ("deep", level), cx.PREC_CELL32)
    world, a_world = _angles(cv, cams, ("deep", level), cx.PREC_WORLD32)
    assert max_err(mixed, ref) <= TOL
    # the cell-local walk: within the paper's bound, here with D >= s (eye about 2.4 cells away)
    e0 = math.sqrt(3) * 2.0 ** -25 * s
    bound = math.degrees(math.asin(min(1.0, math.sqrt(2) * (e0 / s + 7.5 * EPS))))
    assert np.max(a_cell) <= bound
    # canvas coordinates: the eye and positions snap to FP32 values far coarser than the scene
    assert np.max(a_world) > 100 * np.max(a_cell)
    assert max_err(world, ref) > max_err(cell, ref)
    # binary16 cell-local walk: the bound with eps = 2^-10 holds at this depth as well
    _, a16 = _angles(cv, cams, ("deep", level), cx.PREC_CELL16)
    e0_16 = math.sqrt(3) * 2.0 ** -12 * s
    bound16 = math.degrees(math.asin(min(1.0, math.sqrt(2) * (e0_16 / s + 7.5 * EPS16))))
    assert np.all(np.isfinite(a16)) and np.max(a16) <= bound16


@pytest.mark.parametrize("prec,cell_local", [(cx.PREC_CELL32, True), (cx.PREC_WORLD32, False)])
def test_fp32_walks_match_the_oracle_walk(prec, cell_local):
    """The GPU's FP32 walks against the oracle's (the same steps of Sec. 6.2 in FP32 on the CPU), run to the canvas
    exit: the leaves visited per pixel agree exactly, the final angle to float rounding (and 1e-13 deg)."""
    for key, cv, cams in (("c0", config_canvas(0), synth.config_cameras(0, res_scale=0.5)),
                          (("deep", 23),) + _deep_views(23)):
        n = synth.total_pixels(cams)
        steps = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        ang = torch.full((n,), float("nan"), device="cuda")
        render(cv, cams, key=key, precision=prec, t_min=0.0, step_count=steps, angle_deg=ang)
        ref_steps, ref_ang = oracle.walk32(cv, cams, cell_local=cell_local)
        np.testing.assert_array_equal(steps.cpu().numpy(), ref_steps)
        # the final angle is evaluated in FP64 from a cross product that cancels for tiny angles; the compilers
        # contract its products differently, which moves it by about 2^-52 rad (1e-14 deg) at most
        np.testing.assert_allclose(ang.cpu().numpy().astype(np.float64), ref_ang.astype(np.float32).astype(np.float64),
                                   rtol=2.0 ** -22, atol=1e-13)


def _deep_views(level):
    cv, lo, s = _embedded_scene(level)
    centre = lo + 0.5 * s
    cams = synth.cameras_array([
        synth.look_at_camera(centre + np.array([1.3, 0.7, -1.9]) * s, centre, [0, 1, 0], 0.5, 48, 40, 0)])
    return cv, cams
