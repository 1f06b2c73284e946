"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, on a GPU.

The bar is a max abs error of 1e-5 per channel (tests/gpu_util.TOL) for the
mixed-precision and plain FP64 kernels, element by element on the same seeded
inputs. Full images at sizes the oracle finishes in seconds; at the full
benchmark size (c2, 2 x 2160^2 at depth 24) a seeded sample of pixels plus
whole 64x64 tiles. The canvas-coordinate FP32 kernel is expected to fail the
bar at depth >= 24 (Sec. 6.3).
"""
import math

import numpy as np
import pytest

import oracle
import paper_1704_02724_gb300 as cx
from paper_1704_02724_gb300 import canvox
import synth
from synth import random_tree as rt
from gpu_util import TOL, config_canvas, max_err, render, upload
from camera_cases import skewed_cameras

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1704_02724_gb300 import _build
    _build.build()
    assert torch.cuda.is_available()


def test_upload_hash_bit_identity():
    cv = config_canvas(0)
    upload(cv, "c0")
    h, d = cx.octree_hash()
    assert h == d != 0


def test_c0_full_image_mixed_and_fp64():
    cv = config_canvas(0)
    cams = synth.config_cameras(0)
    ref, ic, _ = oracle.render(cv, cams, counters=True)
    steps = torch.zeros(synth.total_pixels(cams), dtype=torch.int32, device="cuda")
    img, st = render(cv, cams, key="c0", step_count=steps)
    assert max_err(img, ref) <= TOL
    # the leaf sequence is the oracle's: per-pixel leaf counts and aggregate reads
    sc = steps.cpu().numpy()
    assert np.mean(sc == ic[:, 0]) > 0.999
    assert abs(st["steps"] - ic[:, 0].sum()) <= 1e-4 * ic[:, 0].sum()
    assert abs(st["slot_reads"] - ic[:, 1].sum()) <= 1e-4 * ic[:, 1].sum()
    assert abs(st["leaf_loads"] - ic[:, 2].sum()) <= 1e-4 * ic[:, 2].sum()
    assert st["rays"] == 256 * 256
    img64, st64 = render(cv, cams, key="c0", precision=cx.PREC_FP64)
    assert max_err(img64, ref) <= 1e-6


def _edge_cameras(extent):
    E = extent
    cams = []
    off = 0

    def add(eye, tgt, w, h, tan=0.6, up=(0, 1, 0), bg=(0.1, 0.2, 0.3, 1)):
        nonlocal off
        cams.append(synth.look_at_camera(np.array(eye) * E, np.array(tgt) * E, up, tan, w, h, off, bg))
        off += w * h + 3   # gaps between views stay unwritten
    add([1.7, 0.4, -1.1], [0.02, -0.03, 0.01], 37, 23)           # ragged tiles
    add([0.1, 0.05, -0.2], [0.3, 0.1, 0.4], 16, 12, tan=1.0)       # eye inside the canvas
    add([0.0, 0.0, 2.0], [0.0, 0.0, 0.0], 9, 9, tan=0.3)           # axis-aligned: zero direction components
    add([0.25, 0.25, 1.5], [0.25, 0.25, 0.0], 5, 5, tan=0.2)       # on cell planes, axis-aligned
    add([2.0, 2.0, 2.0], [0.0, 0.0, 0.0], 1, 1)                    # single pixel through a corner
    add([3.0, 5.0, 0.0], [3.3, 6.0, 0.2], 8, 4)                    # looks away: all background
    add([0.25, 0.0, 0.125], [0.4, 0.3, 0.33], 12, 10, tan=1.2)     # eye inside, exactly on three cell planes
    return synth.cameras_array(cams)


@pytest.mark.parametrize("seed,depth,extent", [(1, 5, 1.0), (2, 6, 3.0), (3, 7, 1000.0), (4, 4, 40000.0)])
def test_random_trees_edge_cameras(seed, depth, extent):
    cv = rt.random_tree(depth, seed=500 + seed, p_refine=0.5, extent=extent)
    cams = _edge_cameras(extent)
    ref = oracle.render(cv, cams)
    written = ~np.isnan(ref[:, 0])
    for prec, tol in ((cx.PREC_MIXED, TOL), (cx.PREC_FP64, 1e-6)):
        img, st = render(cv, cams, key=("rt", seed), precision=prec)
        assert np.all(np.isnan(img[~written]))            # nothing outside the views is touched
        assert max_err(img[written], ref[written]) <= tol, prec


def test_skewed_camera_frames():
    """Cameras whose right/up/forward are not orthonormal (scaled, skewed, a right that points left):
    the library orthonormalises them as the camera model states (forward, then up, then right), so the
    image matches the oracle and equals, within the bar, the render of the frames orthonormalised by
    hand (Sec. 6.1: the FP64 eye frame)."""
    cv = rt.random_tree(6, seed=72, p_refine=0.55, extent=40.0)
    skew, ortho = skewed_cameras(extent=40.0)
    ref = oracle.render(cv, skew)
    for prec, tol in ((cx.PREC_MIXED, TOL), (cx.PREC_FP64, 1e-6)):
        img, _ = render(cv, skew, key="skew", precision=prec)
        assert max_err(img, ref) <= tol, prec
        img_o, _ = render(cv, ortho, key="skew", precision=prec)
        assert max_err(img, img_o) <= tol, prec


@pytest.mark.parametrize("seed,depth,extent", [(1, 5, 1.0), (3, 7, 1000.0), (4, 4, 40000.0)])
def test_fp64_links_twin_random_trees(seed, depth, extent):
    """The FP64 twin of the mixed traversal (same neighbour links and queue, FP64 arithmetic) against the
    oracle at 1e-6 on the edge cameras. (Leaf counts are compared on c0 below: these views put rays on cell
    planes and through edges, where the twin's product form M inv + nod and the oracle's (M - o) / d round
    differently and may add or drop zero-length segments, which change no pixel.)"""
    cv = rt.random_tree(depth, seed=500 + seed, p_refine=0.5, extent=extent)
    cams = _edge_cameras(extent)
    ref = oracle.render(cv, cams)
    written = ~np.isnan(ref[:, 0])
    img, st = render(cv, cams, key=("rt", seed), precision=cx.PREC_FP64_LINKS)
    assert np.all(np.isnan(img[~written]))
    assert max_err(img[written], ref[written]) <= 1e-6
    assert st["rays"] == int(written.sum()) and st["status"] == 0


def test_fp64_links_twin_c0_and_deep_scene():
    """The FP64 twin on the c0 canvas (full image, counters against the oracle's) and on a scene embedded at
    depth 26 of a 40 km canvas, where canvas-coordinate FP32 fails."""
    cv = config_canvas(0)
    cams = synth.config_cameras(0)
    ref, ic, _ = oracle.render(cv, cams, counters=True)
    img, st = render(cv, cams, key="c0", precision=cx.PREC_FP64_LINKS)
    assert max_err(img, ref) <= 1e-6
    assert abs(st["steps"] - ic[:, 0].sum()) <= 1e-4 * ic[:, 0].sum()
    assert abs(st["slot_reads"] - ic[:, 1].sum()) <= 1e-4 * ic[:, 1].sum()
    cv, lo, s = _embedded_scene(26)
    centre = lo + 0.5 * s
    cams = synth.cameras_array([
        synth.look_at_camera(centre + np.array([1.7, 0.6, -1.3]) * s, centre, [0, 1, 0], 0.7, 48, 40, 0,
                             (0.1, 0.2, 0.3, 1.0)),
        synth.look_at_camera(centre + np.array([0.1, -0.2, 0.15]) * s, centre + np.array([0.4, 0.3, 0.2]) * s,
                             [0, 1, 0], 1.0, 32, 32, 48 * 40, (0.1, 0.2, 0.3, 1.0))])
    ref = oracle.render(cv, cams)
    img, _ = render(cv, cams, key=("deep", 26), precision=cx.PREC_FP64_LINKS)
    assert max_err(img, ref) <= 1e-6


def test_t_min_zero_runs_to_canvas_exit():
    cv = rt.random_tree(6, seed=77, p_refine=0.55, sigma_range=(0.5, 30.0))
    cams = _edge_cameras(1.0)
    ref = oracle.render(cv, cams, t_min=0.0)
    w = ~np.isnan(ref[:, 0])
    img, _ = render(cv, cams, key="t0", t_min=0.0)
    assert max_err(img[w], ref[w]) <= TOL


def _embedded_scene(level):
    """A depth-4 random scene as one cell at `level` of a 40 km canvas (cell side 40000 * 2^-level)."""
    small = rt.random_nested(4, seed=91, p_refine=0.6, sigma_range=(0.5, 20.0))
    E = 40000.0
    cell = (2 ** (level - 1) + 12345, 2 ** (level - 1) - 777, 2 ** (level - 2) + 5)
    s = E * 2.0 ** -level
    # extinction per metre so that the scene has the same optical depth per cell side
    def scale(t):
        if isinstance(t, list):
            return [scale(c) for c in t]
        if t is None:
            return None
        return (t[0], t[1], t[2], t[3] / s)
    big = rt.from_nested(rt.embed(scale(small), 4, level, cell), level + 4, E)
    lo = np.array([-0.5 * E + c * s for c in cell])
    return big, lo, s


@pytest.mark.parametrize("level", [20, 23, 26])
def test_deep_embedding_mixed_passes_fp32_fails(level):
    cv, lo, s = _embedded_scene(level)
    centre = lo + 0.5 * s
    cams = synth.cameras_array([
        synth.look_at_camera(centre + np.array([1.3, 0.7, -1.9]) * s, centre, [0, 1, 0], 0.5, 48, 40, 0),
        synth.look_at_camera(centre + np.array([0.1, -0.2, 0.15]) * s, centre + np.array([0.4, 0.3, -0.2]) * s,
                             [0, 1, 0], 1.0, 32, 32, 48 * 40),
    ])
    ref = oracle.render(cv, cams)
    img, _ = render(cv, cams, key=("deep", level))
    assert max_err(img, ref) <= TOL
    if level >= 23:
        img32, _ = render(cv, cams, key=("deep", level), precision=cx.PREC_FP32)
        assert max_err(img32, ref) > 1e-3   # canvas-coordinate FP32 drifts at this depth


@pytest.mark.parametrize("level,frames", [(23, 20), (26, 3), (26, 22)])
def test_axis_aligned_rays_in_deep_frames(level, frames):
    """Rays with one or two zero direction components (the middle row and column of odd-sized views whose
    forward axis is a canvas axis), eyes on the scene's cell planes, inside the scene embedded deep in a
    40 km canvas: such an axis has no crossing time, and the ray's fixed coordinate on it decides every child
    side on that axis through frame set-ups, rebases and descents (Sec. 6.2's cell-local frames)."""
    cv, lo, s = _embedded_scene(level)
    bg = (0.1, 0.2, 0.3, 1.0)
    e1 = lo + np.array([0.5, 0.25, 1.7]) * s        # on the x mid-plane and a y quarter plane, looking down -z
    e2 = lo + np.array([-0.6, 0.5, 0.375]) * s      # outside the scene, looking along +x through it
    e3 = lo + np.array([0.1, 0.625, 0.5]) * s       # inside the scene, looking along +y
    cams = synth.cameras_array([
        synth.look_at_camera(e1, e1 - np.array([0.0, 0.0, 1.0]) * s, [0, 1, 0], 0.4, 9, 9, 0, bg),
        synth.look_at_camera(e2, e2 + np.array([1.0, 0.0, 0.0]) * s, [0, 1, 0], 0.3, 7, 5, 81, bg),
        synth.look_at_camera(e3, e3 + np.array([0.0, 1.0, 0.0]) * s, [0, 0, 1], 0.9, 11, 9, 81 + 35, bg)])
    ref = oracle.render(cv, cams)
    img, st = render(cv, cams, key=("deep", level), frame_levels=frames)
    assert max_err(img, ref) <= TOL
    assert st["status"] == 0 and st["rays"] == 81 + 35 + 99
    img64, _ = render(cv, cams, key=("deep", level), precision=cx.PREC_FP64_LINKS)
    assert max_err(img64, ref) <= 1e-6


@pytest.mark.parametrize("frames,traversal", [(2, 0), (3, 1), (8, 0), (8, 1)])
def test_small_frames_rebase_often(frames, traversal):
    """Frames only a few levels deep make nearly every descent and many crossings rebase the ray (FP64 frame
    set-ups): the images stay within the bar on c0 and on the scene embedded at depth 23, with both traversals."""
    cv, lo, s = _embedded_scene(23)
    centre = lo + 0.5 * s
    deep_cams = synth.cameras_array([
        synth.look_at_camera(centre + np.array([1.3, 0.7, -1.9]) * s, centre, [0, 1, 0], 0.5, 48, 40, 0),
        synth.look_at_camera(centre + np.array([0.1, -0.2, 0.15]) * s, centre + np.array([0.4, 0.3, -0.2]) * s,
                             [0, 1, 0], 1.0, 32, 32, 48 * 40)])
    for key, canvas, cams in ((("deep", 23), cv, deep_cams), ("c0", config_canvas(0), synth.config_cameras(0, 0.5))):
        ref = oracle.render(canvas, cams)
        img, st = render(canvas, cams, key=key, frame_levels=frames, traversal=traversal)
        if key != "c0" or frames < 8:    # (c0 is 8 levels deep: 8-level frames never need a rebase there)
            assert st["rebases"] > st["rays"]
        assert max_err(img, ref) <= TOL, (key, frames, traversal)


@pytest.mark.parametrize("budget", [0.0, 1.0])
def test_error_budget_extremes(budget):
    """err_budget 0 takes every boundary between different leaves in FP64 (the fallback path on every step),
    err_budget 1 never does; both stay within the bar."""
    cv, lo, s = _embedded_scene(26)
    centre = lo + 0.5 * s
    cams = synth.cameras_array([
        synth.look_at_camera(centre + np.array([1.3, 0.7, -1.9]) * s, centre, [0, 1, 0], 0.5, 48, 40, 0)])
    ref = oracle.render(cv, cams)
    img, st = render(cv, cams, key=("deep", 26), err_budget=budget)
    if budget == 0.0:
        assert st["fp64_boundaries"] > st["rays"]
    assert max_err(img, ref) <= TOL


def test_graph_cache_follows_the_view_layout():
    """Graph replay with one view layout, then another, then the first again: every render matches the
    direct launch of the same views (the cached graph is keyed on sizes, offsets, output and options)."""
    cv = config_canvas(0)
    a = _edge_cameras(1.0)
    b = synth.config_cameras(0, res_scale=0.5)
    ref_a, _ = render(cv, a, key="c0")
    ref_b, _ = render(cv, b, key="c0")
    for cams, ref in ((a, ref_a), (b, ref_b), (a, ref_a), (b, ref_b)):
        img, _ = render(cv, cams, key="c0", use_graph=1)
        np.testing.assert_array_equal(img, ref)


def test_root_array_canvas():
    """A canvas whose top two levels are refined everywhere (the 4^3 array of octree roots of Sec. 4):
    the mixed path against the oracle, and the same image as the merged canvas of the same strokes."""
    rng = synth.Rng(170402724)
    n = 400
    U = rng.uniform(n * 8).reshape(n, 8)
    c = 0.02 + 0.46 * U[:, 0:3]                      # strokes in one octant: the others are empty roots
    r = (2.0 + 18.0 * U[:, 3]) / 256.0
    q = np.c_[U[:, 4:7], 0.5 + 19.5 * U[:, 7]].astype(np.float32)
    a = synth.stamp_canvas(8, 1.0, c, r, q)
    b = synth.stamp_canvas(8, 1.0, c, r, q, root_levels=2)
    assert np.all(b.nodes[0] > 0) and b.n_records > a.n_records
    cams = synth.config_cameras(0, res_scale=0.5)
    ref = oracle.render(b, cams)
    img_b, _ = render(b, cams, key="root_array")
    img_a, _ = render(a, cams, key="root_array_merged")
    assert max_err(img_b, ref) <= TOL
    assert max_err(img_a, img_b) <= TOL


def test_c1_reduced_full_image():
    cv = config_canvas(1)
    cams = synth.config_cameras(1, res_scale=0.125)
    ref = oracle.render(cv, cams)
    img, st = render(cv, cams, key="c1")
    assert max_err(img, ref) <= TOL


def _sample_pixels(cams, n_random, n_tiles, seed):
    rng = np.random.default_rng(seed)
    total = synth.total_pixels(cams)
    idx = set(rng.choice(total, size=min(n_random, total), replace=False).tolist())
    for c in cams:
        W, H, off = int(c["width"]), int(c["height"]), int(c["out_offset_px"])
        for _ in range(n_tiles):
            x0, y0 = rng.integers(0, max(1, W - 64)), rng.integers(0, max(1, H - 64))
            for j in range(y0, min(H, y0 + 64)):
                idx.update(range(off + j * W + x0, off + j * W + min(W, x0 + 64)))
    return np.array(sorted(idx), dtype=np.int64)


@pytest.mark.parametrize("cid,n_random", [(1, 100000), (2, 300000), (3, 200000), (4, 200000)])
def test_full_size_sampled(cid, n_random):
    """Full-size images with the built-in schedule and with the one the autotuner picks for these views (the
    schedule bench.py times); oracle on sampled pixels."""
    from gpu_util import _uploaded
    cv = config_canvas(cid)
    cams = synth.config_cameras(cid)
    key = f"c{3 if cid == 4 else cid}"
    px = _sample_pixels(cams, n_random, 2, seed=cid)
    ref = oracle.render(cv, cams, px_idx=px)
    img, st = render(cv, cams, key=key)
    upload(cv, key)
    best = cx.autotune(cams)
    img_tuned, st_tuned = render(cv, cams, key=key, **{k: best[k] for k in ("tile_w", "frame_levels", "traversal")})
    cx.release()                     # back to the built-in schedule for the tests that follow
    _uploaded["key"] = None
    for im, s_ in ((img, st), (img_tuned, st_tuned)):
        assert s_["status"] == 0
        err = np.abs(im[px] - ref)
        assert float(err.max()) <= TOL, (float(err.max()), int(np.sum(err.max(1) > TOL)), best)
        assert np.all(np.isfinite(im))


def test_schedules_agree_bitwise():
    """Schedule options change which lane traces which ray, never a ray's arithmetic.
    (frame_levels changes the frames, hence the rounding; it is checked against the bar instead.)"""
    cv = config_canvas(0)
    cams = _edge_cameras(1.0)
    base, _ = render(cv, cams, key="c0")
    for kw in (dict(per_view=1), dict(use_graph=1), dict(use_graph=1), dict(refill=0, block_threads=128),
               dict(refill=31, blocks_per_sm=1), dict(tile_w=4), dict(tile_w=32, refill=2), dict(tile_w=16),
               dict(smem_records=1024, block_threads=128), dict(smem_records=100),
               dict(smem_records=6144, block_threads=128), dict(traversal=1),
               dict(traversal=1, smem_records=100), dict(traversal=1, per_view=1)):
        img, _ = render(cv, cams, key="c0", **kw)
        np.testing.assert_array_equal(img, base, err_msg=str(kw))


def test_read_counters_off_same_image():
    """count_reads = 0 runs the kernel instance without the per-lane read counters: the same image bit for bit,
    slot reads, leaf loads and record loads reported as 0, the other counters unchanged."""
    cv = config_canvas(0)
    cams = _edge_cameras(1.0)
    a, sa = render(cv, cams, key="c0")
    for kw in (dict(), dict(traversal=1), dict(smem_records=100)):
        b, sb = render(cv, cams, key="c0", count_reads=0, **kw)
        np.testing.assert_array_equal(a, b, err_msg=str(kw))
        assert sb["slot_reads"] == sb["leaf_loads"] == sb["record_loads"] == 0
        assert (sb["rays"], sb["steps"]) == (sa["rays"], sa["steps"])
    assert sa["slot_reads"] > 0 and sa["leaf_loads"] > 0


def test_frame_levels_do_not_change_depth27_pixels():
    """Frames of 1 to 22 levels give the same image within the bar on the depth-27 canvas (precision pin)."""
    cv = config_canvas(3)
    cams = synth.config_cameras(3, res_scale=0.05)
    ref = oracle.render(cv, cams)
    for K in (1, 8, 22):
        img, st = render(cv, cams, key="c3", frame_levels=K)
        assert max_err(img, ref) <= TOL, K


def test_autotune_keeps_results():
    cv = config_canvas(0)
    cams = _edge_cameras(1.0)
    base, _ = render(cv, cams, key="c0")
    best = cx.autotune(cams)
    assert best["tile_w"] in (4, 8, 16, 32) and best["block_threads"] in (128, 256)
    assert cx.default_opts()["tile_w"] == best["tile_w"]
    img, _ = render(cv, cams, key="c0")
    np.testing.assert_array_equal(img, base)


def test_render_host_matches_device():
    cv = config_canvas(0)
    cams = synth.config_cameras(0)
    dev, _ = render(cv, cams, key="c0")
    host = np.zeros((synth.total_pixels(cams), 4), np.float32)
    cx.render_host(cams, host)
    np.testing.assert_array_equal(host.astype(np.float64), dev)


def test_step_limit_reports_status():
    cv = config_canvas(0)
    cams = synth.config_cameras(0)
    img, st = render(cv, cams, key="c0", step_limit=3)
    assert st["status"] == canvox.ERR_STEP_LIMIT and st["step_limited"] > 0
    assert np.all(np.isfinite(img))
    host = np.zeros((synth.total_pixels(cams), 4), np.float32)
    with pytest.raises(cx.CanvoxError) as e:
        cx.render_host(cams, host, step_limit=3)
    assert e.value.code == canvox.ERR_STEP_LIMIT
    img2, st2 = render(cv, cams, key="c0")   # the next render starts clean
    assert st2["status"] == 0


def test_empty_canvas_zero_views_and_bad_cameras():
    cv = rt.from_nested([None] * 8, 1, 40000.0)
    cams = _edge_cameras(40000.0)
    img, st = render(cv, cams, key="empty")
    ref = oracle.render(cv, cams)
    w = ~np.isnan(ref[:, 0])
    assert np.array_equal(img[w].astype(np.float32), ref[w].astype(np.float32))
    out = torch.zeros((4, 4), device="cuda")
    cx.render(cams[:0], out)          # no views: no-op
    bad = cams.copy()
    bad[0]["width"] = 0
    with pytest.raises(cx.CanvoxError) as e:
        cx.render(bad, out)
    assert e.value.code == canvox.ERR_INVALID_ARG
    bad = cams.copy()
    bad[1]["tan_half_fov_y"] = math.nan
    with pytest.raises(cx.CanvoxError):
        cx.render(bad, out)
    bad = cams.copy()
    bad[0]["width"], bad[0]["height"] = 65536, 32768   # 2^31 pixels: beyond the per-view limit
    with pytest.raises(cx.CanvoxError) as e:
        cx.render(bad, out)
    assert e.value.code == canvox.ERR_INVALID_ARG


def test_update_leaves_equals_full_upload():
    """A value edit uploaded as a dirty leaf range renders (bit for bit) and hashes like the edited pools
    uploaded whole; a bad range or value changes nothing."""
    cv = config_canvas(0)
    cams = synth.config_cameras(0, res_scale=0.5)
    edited = cv.leaves.copy()
    lo, hi = 100_000, 140_000
    vals = edited[lo:hi].view(np.float16).astype(np.float32)
    vals[:, 0:3] = vals[:, [2, 0, 1]]          # recolour
    vals[:, 3] *= 0.25                          # thinner paint
    edited[lo:hi] = vals.astype(np.float16).view(np.uint16)
    upload(cv, "c0")
    cx.update_leaves(lo, edited[lo:hi])
    h, d = cx.octree_hash()
    assert h == d
    img, _ = render(cv, cams, key="c0")         # the cached upload, edited in place
    with pytest.raises(cx.CanvoxError) as e:
        cx.update_leaves(cv.n_leaves - 1, edited[:2])
    assert e.value.code == canvox.ERR_INVALID_ARG
    bad = edited[lo:lo + 1].copy()
    bad[0, 3] = np.float16(-1.0).view(np.uint16)
    with pytest.raises(cx.CanvoxError) as e:
        cx.update_leaves(lo, bad)
    assert e.value.code == canvox.ERR_BAD_TREE
    assert cx.octree_hash() == (h, d)
    whole = synth.Canvas(nodes=cv.nodes, leaves=edited, depth=cv.depth, extent=cv.extent, levels=cv.levels, info={})
    ref, _ = render(whole, cams, key="c0_edited_whole")
    np.testing.assert_array_equal(img, ref)
    assert cx.octree_hash() == (h, d)
    assert max_err(img, oracle.render(whole, cams)) <= TOL


def test_bad_upload_keeps_previous_canvas():
    cv = config_canvas(0)
    upload(cv, "c0")
    bad = cv.nodes.copy()
    bad[0, 0] = 7
    with pytest.raises(cx.CanvoxError):
        cx.upload_octree(bad, cv.leaves, cv.depth, cv.extent)
    cams = synth.config_cameras(0, res_scale=0.25)
    img, _ = render(cv, cams, key="c0")
    assert max_err(img, oracle.render(cv, cams)) <= TOL
