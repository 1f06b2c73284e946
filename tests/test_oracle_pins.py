"""Pins of the FP64 oracle against things other than itself (CPU only).

* a brute-force uniform-grid marcher (tests/bruteforce.py) on random trees,
  for pixels, leaf counts and perfect-stack slot reads;
* a hand-derived worked example (tests/golden/worked_example_depth1.json);
* closed forms: homogeneous cube 1 - exp(-sigma L), empty canvas = background;
* invariants: coarsening, mirror symmetry, embedding at depth 20+ (the
  precision claim of Sec. 6.1-6.3 holds exactly for an FP64 oracle);
* the camera model: pixel rays recomputed independently, and the orthonormalisation of
  skewed camera frames against a numpy restatement.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth
from synth import random_tree as rt
from bruteforce import DenseGrid, march
from camera_cases import gram_schmidt, skewed_cameras

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _random_rays(seed, n, extent, inside_frac=0.3):
    rng = np.random.default_rng(seed)
    o = np.empty((n, 3))
    d = rng.normal(size=(n, 3))
    for i in range(n):
        if rng.random() < inside_frac:
            o[i] = rng.uniform(-0.5, 0.5, 3) * extent
        else:
            # outside, aimed at a random point inside
            o[i] = rng.normal(size=3)
            o[i] *= 1.6 * extent / np.linalg.norm(o[i])
            d[i] = rng.uniform(-0.45, 0.45, 3) * extent - o[i]
    return o, d


@pytest.mark.parametrize("seed,depth", [(1, 3), (2, 4), (3, 5), (4, 5), (5, 6), (6, 4)])
def test_bruteforce_random_trees(seed, depth):
    cv = rt.random_tree(depth, seed=1000 + seed, p_refine=0.5, extent=[1.0, 3.0, 1000.0][seed % 3])
    grid = DenseGrid(cv)
    o, d = _random_rays(seed, 120, cv.extent)
    bg = (0.2, 0.5, 0.7, 1.0)
    got, ic, _ = oracle.trace_rays(cv, o, d, bg, t_min=0.0, counters=True)
    for i in range(o.shape[0]):
        ref, steps, reads = march(grid, o[i], d[i], bg)
        np.testing.assert_allclose(got[i], ref, rtol=0, atol=1e-12)
        assert ic[i, 0] == steps
        assert ic[i, 1] == reads


def test_bruteforce_axis_aligned_and_on_planes():
    """Directions with zero components and origins on cell planes (tie conventions)."""
    cv = rt.random_tree(5, seed=77, p_refine=0.55)
    grid = DenseGrid(cv)
    w = 1.0 / 32
    rng = np.random.default_rng(5)
    rays = []
    for _ in range(150):
        o = rng.integers(-16, 16, 3) * w + rng.choice([0.0, 0.5 * w, 0.25 * w], 3)
        d = rng.choice([-1.0, 0.0, 1.0, 0.5], 3)
        if not d.any():
            d[rng.integers(3)] = 1.0
        axis = rng.integers(3)
        o[axis] = rng.choice([-1.5, 1.5]) if rng.random() < 0.5 else o[axis]
        rays.append((o, d))
    o = np.array([r[0] for r in rays])
    d = np.array([r[1] for r in rays])
    got = oracle.trace_rays(cv, o, d, (0.3, 0.3, 0.3, 1.0), t_min=0.0)
    for i in range(len(rays)):
        ref, _, _ = march(grid, o[i], d[i], (0.3, 0.3, 0.3, 1.0))
        np.testing.assert_allclose(got[i], ref, rtol=0, atol=1e-12)


def test_golden_worked_example():
    with open(os.path.join(GOLDEN, "worked_example_depth1.json")) as f:
        g = json.load(f)
    tree = [None] * 8
    for k, v in g["leaves"].items():
        tree[int(k)] = tuple(v)
    cv = rt.from_nested(tree, g["depth"], g["extent"])
    bg = [float(x) for x in np.asarray(g["background"], dtype=np.float32)]
    for ray in g["rays"]:
        C = [0.0, 0.0, 0.0]
        T = 1.0
        for k, L in ray["segments"]:
            if str(k) in g["leaves"]:
                r, gg, b, s = g["leaves"][str(k)]
                a = 1.0 - math.exp(-s * L)
                C = [C[0] + T * a * r, C[1] + T * a * gg, C[2] + T * a * b]
                T *= math.exp(-s * L)
        expect = [C[0] + T * bg[0], C[1] + T * bg[1], C[2] + T * bg[2], 1.0 - T]
        got = oracle.trace_rays(cv, [ray["o"]], [ray["d"]], bg, t_min=0.0)[0]
        np.testing.assert_allclose(got, expect, rtol=0, atol=1e-15, err_msg=ray["why"])


@pytest.mark.parametrize("depth", [1, 5])
def test_homogeneous_cube_closed_form(depth):
    """rgb = c (1 - e^{-sigma L}) + bg e^{-sigma L}, L = slab chord, for any refinement of a uniform cube."""
    value = (0.75, 0.5, 0.125, 3.5)   # exact in FP16
    cv = rt.uniform_tree(depth, value, extent=2.0)
    o, d = _random_rays(11, 200, 2.0)
    bg = [float(x) for x in np.float32([0.1, 0.2, 0.3, 1.0])]
    got = oracle.trace_rays(cv, o, d, bg, t_min=0.0)
    for i in range(o.shape[0]):
        dn = d[i] / np.linalg.norm(d[i])
        t0, t1 = 0.0, math.inf
        for a in range(3):
            if dn[a] != 0:
                ta, tb = (-1 - o[i, a]) / dn[a], (1 - o[i, a]) / dn[a]
                t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
        L = max(0.0, t1 - t0)
        Tr = math.exp(-value[3] * L)
        expect = [value[c] * (1 - Tr) + bg[c] * Tr for c in range(3)] + [1 - Tr]
        np.testing.assert_allclose(got[i], expect, rtol=0, atol=1e-13)


def test_empty_canvas_is_background():
    cv = rt.from_nested([None] * 8, 1, 40000.0)
    cams = synth.cameras_array([synth.look_at_camera([3e4, 1e4, -2e4], [0, 0, 0], [0, 1, 0], 0.7, 17, 9, 0,
                                                     (0.25, 0.5, 0.125, 1.0))])
    img = oracle.render(cv, cams)
    assert np.array_equal(img, np.tile([0.25, 0.5, 0.125, 0.0], (17 * 9, 1)))


def test_coarsening_invariance():
    """A leaf and the same leaf split into eight identical children render the same."""
    nested = rt.random_nested(4, seed=31, p_refine=0.5)

    def split_some(t, rng):
        if not isinstance(t, list):
            return t
        out = []
        for c in t:
            if not isinstance(c, list) and rng.random() < 0.4:
                out.append([c] * 8)
            else:
                out.append(split_some(c, rng))
        return out

    fine = split_some(nested, np.random.default_rng(3))
    a = rt.from_nested(nested, 4, 1.0)
    b = rt.from_nested(fine, 5, 1.0)
    o, d = _random_rays(21, 300, 1.0)
    ra = oracle.trace_rays(a, o, d, (0.5, 0.5, 0.5, 1), t_min=0.0)
    rb = oracle.trace_rays(b, o, d, (0.5, 0.5, 0.5, 1), t_min=0.0)
    np.testing.assert_allclose(ra, rb, rtol=0, atol=1e-13)


def test_mirror_symmetry():
    nested = rt.random_nested(5, seed=41, p_refine=0.5)
    a = rt.from_nested(nested, 5, 1.0)
    b = rt.from_nested(rt.mirror_x(nested), 5, 1.0)
    o, d = _random_rays(22, 300, 1.0)
    om, dm = o.copy(), d.copy()
    om[:, 0] *= -1
    dm[:, 0] *= -1
    ra = oracle.trace_rays(a, o, d, (0.1, 0.1, 0.1, 1), t_min=0.0)
    rb = oracle.trace_rays(b, om, dm, (0.1, 0.1, 0.1, 1), t_min=0.0)
    np.testing.assert_allclose(ra, rb, rtol=0, atol=1e-14)


@pytest.mark.parametrize("level", [20, 24])
def test_embedding_invariance_deep(level):
    """A depth-4 scene rendered alone and as one cell at depth 20-24 of a huge canvas (cell size 1)."""
    small = rt.random_nested(4, seed=51, p_refine=0.6)
    a = rt.from_nested(small, 4, 1.0)
    E = float(2 ** level)
    cell = (2 ** (level - 1) + 12345 % 2 ** (level - 1), 2 ** (level - 2) + 7, 3)
    big = rt.from_nested(rt.embed(small, 4, level, cell), level + 4, E)
    off = np.array([-0.5 * E + c + 0.5 for c in cell])
    rng = np.random.default_rng(8)
    # dyadic origins and directions, so the shifted origins are exact in FP64
    o = np.round(rng.uniform(-1.5, 1.5, (300, 3)) * 2 ** 20) / 2 ** 20
    tgt = np.round(rng.uniform(-0.45, 0.45, (300, 3)) * 2 ** 20) / 2 ** 20
    d = tgt - o
    ra = oracle.trace_rays(a, o, d, (0, 0, 0, 0), t_min=0.0)
    rb = oracle.trace_rays(big, o + off, d, (0, 0, 0, 0), t_min=0.0)
    np.testing.assert_allclose(ra, rb, rtol=0, atol=1e-13)


def test_termination_threshold_bound():
    """Stopping at T < T_min changes a pixel by at most T_min (remaining light <= T max(rgb, bg) <= T)."""
    cv = rt.random_tree(5, seed=61, p_refine=0.5, sigma_range=(20.0, 200.0))
    o, d = _random_rays(23, 300, 1.0)
    full = oracle.trace_rays(cv, o, d, (1, 1, 1, 1), t_min=0.0)
    cut = oracle.trace_rays(cv, o, d, (1, 1, 1, 1), t_min=2.0 ** -8)
    assert np.max(np.abs(full - cut)) <= 2.0 ** -8
    assert np.max(np.abs(full - cut)) > 0


def test_camera_pixel_rays():
    """render() = trace_rays() over pixel-centre rays d = f + u r + v up (vertical FOV, square pixels)."""
    cv = rt.random_tree(5, seed=71, p_refine=0.5)
    eye = np.array([1.3, 0.4, -1.7])
    cam = synth.look_at_camera(eye, [0.05, -0.02, 0.1], [0, 1, 0], math.tan(math.radians(35)), 23, 11, 5,
                               (0.1, 0.2, 0.3, 1))
    cams = synth.cameras_array([cam])
    img = oracle.render(cv, cams)
    assert img.shape == (5 + 23 * 11, 4)
    assert np.all(np.isnan(img[:5]))
    W, H, t = 23, 11, float(cam["tan_half_fov_y"])
    f, r, u = cam["forward"], cam["right"], cam["up"]
    dirs = []
    for j in range(H):
        for i in range(W):
            x = (2 * (i + 0.5) / W - 1) * t * W / H
            y = (1 - 2 * (j + 0.5) / H) * t
            dirs.append(f + x * r + y * u)
    ref = oracle.trace_rays(cv, np.tile(eye, (W * H, 1)), np.array(dirs), (0.1, 0.2, 0.3, 1))
    np.testing.assert_allclose(img[5:], ref, rtol=0, atol=1e-12)


def test_camera_gram_schmidt_on_skewed_frames():
    """A non-orthonormal camera renders exactly like its frame orthonormalised by hand in the camera
    model's order (forward, then up, then right); the other orders give other images (Sec. 6.1:
    the FP64 eye frame that every pixel ray is built from)."""
    cv = rt.random_tree(5, seed=72, p_refine=0.55)
    skew, ortho = skewed_cameras()
    got = oracle.render(cv, skew)
    ref = oracle.render(cv, ortho)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)
    assert np.mean(np.abs(ref[:, 3]) > 0) > 0.3    # the views see paint
    # an up-first order, or a right that is only made orthogonal to forward, moves the image: the
    # pixel rays of those frames (traced as given, not orthonormalised again) differ from the pin
    for c in skew:
        W, H, t = int(c["width"]), int(c["height"]), float(c["tan_half_fov_y"])
        o, n = int(c["out_offset_px"]), W * H
        u = c["up"] / np.linalg.norm(c["up"])
        f = c["forward"] - (c["forward"] @ u) * u
        f /= np.linalg.norm(f)
        r = c["right"] - (c["right"] @ f) * f - (c["right"] @ u) * u
        r /= np.linalg.norm(r)
        f2, u2, _ = gram_schmidt(c["forward"], c["up"], c["right"])
        r2 = c["right"] - (c["right"] @ f2) * f2
        r2 /= np.linalg.norm(r2)
        for fw, uw, rw in ((f, u, r), (f2, u2, r2)):
            dirs = [fw + ((2 * (i + 0.5) / W - 1) * t * W / H) * rw + ((1 - 2 * (j + 0.5) / H) * t) * uw
                    for j in range(H) for i in range(W)]
            bad = oracle.trace_rays(cv, np.tile(c["eye"], (n, 1)), np.array(dirs), tuple(c["background"]))
            assert np.max(np.abs(bad - ref[o:o + n])) > 1e-3


def test_stamp_canvas_matches_bruteforce():
    """The oracle on a stroke-built canvas (the real workload kind) vs the dense grid."""
    rng = synth.Rng(99)
    n = 40
    U = rng.uniform(n * 8).reshape(n, 8)
    c = -0.5 + U[:, 0:3]
    r = (1.0 + 6.0 * U[:, 3]) / 32.0
    q = np.c_[U[:, 4:7], 0.5 + 19.5 * U[:, 7]].astype(np.float32)
    cv = synth.stamp_canvas(5, 1.0, c, r, q)
    grid = DenseGrid(cv)
    o, d = _random_rays(24, 150, 1.0)
    got, ic, _ = oracle.trace_rays(cv, o, d, (0, 0, 0, 0), t_min=0.0, counters=True)
    for i in range(o.shape[0]):
        ref, steps, reads = march(grid, o[i], d[i])
        np.testing.assert_allclose(got[i], ref, rtol=0, atol=1e-12)
        assert (ic[i, 0], ic[i, 1]) == (steps, reads)


def test_footprint_matches_bruteforce():
    """The records and stored leaves the oracle marks = the root-to-leaf paths of the leaves the dense-grid
    marcher enters (no tree descent there), over every pixel of a view."""
    cv = rt.random_tree(5, seed=41, p_refine=0.5)
    eye = np.array([1.1, -0.6, 1.5])
    cam = synth.look_at_camera(eye, [0.02, 0.07, -0.04], [0, 1, 0], math.tan(math.radians(30)), 21, 13, 0,
                               (0, 0, 0, 1))
    cams = synth.cameras_array([cam])
    rm, lm, img = oracle.footprint(cv, cams, t_min=0.0)
    np.testing.assert_allclose(img, oracle.render(cv, cams, t_min=0.0), rtol=0, atol=0)
    grid = DenseGrid(cv)
    W, H, t = 21, 13, float(cam["tan_half_fov_y"])
    f, r, u = cam["forward"], cam["right"], cam["up"]
    rec_ref = np.zeros(cv.nodes.shape[0], dtype=bool)
    leaf_ref = np.zeros(cv.n_leaves, dtype=bool)
    for j in range(H):
        for i in range(W):
            x = (2 * (i + 0.5) / W - 1) * t * W / H
            y = (1 - 2 * (j + 0.5) / H) * t
            seen = []
            march(grid, eye, f + x * r + y * u, visited=seen)
            for lid in seen:
                rec = 0
                for k in grid.paths[lid]:
                    rec_ref[rec] = True
                    v = int(cv.nodes[rec, k])
                    if v > 0:
                        rec = v
                    elif v < 0:
                        leaf_ref[-v - 1] = True
    assert rec_ref.sum() > 10 and leaf_ref.sum() > 10
    np.testing.assert_array_equal(rm, rec_ref)
    np.testing.assert_array_equal(lm, leaf_ref)


def test_walk32_axis_aligned_rays_are_exact():
    """The paper's FP32 walks on rays along an axis from dyadic points: every FP32 quantity is exact, so both
    walks visit exactly the FP64 oracle's leaves and end on the axis (angle 0)."""
    cv = rt.random_tree(6, seed=303, p_refine=0.55)
    cams = []
    off = 0
    for eye, tgt in (([0.125, 0.3125, 1.5], [0.125, 0.3125, 0.0]), ([-2.0, 0.0625, -0.1875], [0.0, 0.0625, -0.1875]),
                     ([0.4375, -1.75, 0.25], [0.4375, 0.0, 0.25])):
        c = synth.look_at_camera(eye, tgt, [1, 0, 0] if eye[1] == -1.75 else [0, 1, 0], 0.3, 1, 1, off)
        cams.append(c)
        off += 1
    cams = synth.cameras_array(cams)
    _, ic, _ = oracle.render(cv, cams, t_min=0.0, counters=True)
    for cell in (True, False):
        st, an = oracle.walk32(cv, cams, cell_local=cell)
        np.testing.assert_array_equal(st, ic[:, 0])
        assert np.all(an == 0.0)


def test_walk32_within_the_paper_bound():
    """Cell-local FP32 walk (Sec. 6.2) on a general view: the ray-angle error stays within the paper's bound
    asin(sqrt(2)(e0/L + 7.5 eps)) (Sec. 6.3), and the walk visits the FP64 oracle's leaves on almost every pixel."""
    cv = synth.build_config(0)
    cams = synth.config_cameras(0, res_scale=0.5)
    _, ic, _ = oracle.render(cv, cams, t_min=0.0, counters=True)
    st, an = oracle.walk32(cv, cams, cell_local=True)
    hit = ic[:, 0] > 0
    assert np.mean(st[hit] == ic[hit, 0]) > 0.99
    eps = 2.0 ** -23
    e0 = math.sqrt(3) * 2.0 ** -25 * 0.5
    assert np.max(an) <= math.degrees(math.asin(math.sqrt(2) * (e0 / 1.5 + 7.5 * eps)))
    st_w, an_w = oracle.walk32(cv, cams, cell_local=False)
    assert np.max(an_w) > np.max(an)


def test_leaf_numbers_are_the_breadth_first_slot_rank():
    """Stored leaves are numbered 0, 1, ... in breadth-first slot order (Sec. 4.1.1's index pools), and the slot
    holds the number modulo 2^31. The generator's pools: -slot-1 is that rank for every leaf slot (canvases
    below 2^31 leaves). The oracle's per-record base equals a numpy prefix count, and the oracle reads leaves
    by the rank alone: pools whose leaf slots all hold -1 render identically."""
    cv = synth.stamp_canvas(6, 1.0, *[a for a in _stamps(7)])
    neg = cv.nodes < 0
    rank = np.cumsum(neg.ravel()) - 1
    np.testing.assert_array_equal((-cv.nodes.ravel()[neg.ravel()] - 1), rank[neg.ravel()])
    base = np.empty(cv.n_records, dtype=np.int64)
    oracle.lib().oracle_leaf_base(np.ascontiguousarray(cv.nodes).ctypes.data, cv.n_records, base.ctypes.data)
    np.testing.assert_array_equal(base, np.concatenate([[0], np.cumsum(neg.sum(axis=1))[:-1]]))
    blind = synth.Canvas(nodes=np.where(neg, -1, cv.nodes).astype(np.int32), leaves=cv.leaves, depth=cv.depth,
                         extent=cv.extent)
    o, d = _random_rays(31, 300, 1.0)
    np.testing.assert_array_equal(oracle.trace_rays(cv, o, d, (0.2, 0.3, 0.4, 1)),
                                  oracle.trace_rays(blind, o, d, (0.2, 0.3, 0.4, 1)))


def _stamps(seed, n=60):
    rng = synth.Rng(seed)
    U = rng.uniform(n * 8).reshape(n, 8)
    return -0.5 + U[:, 0:3], (1.0 + 6.0 * U[:, 3]) / 64.0, np.c_[U[:, 4:7], 0.5 + 19.5 * U[:, 7]].astype(np.float32)
