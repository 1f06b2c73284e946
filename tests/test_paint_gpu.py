"""The device-side stamp painter (Sec. 5.1-5.2 on the GPU) against the host painter of the input
generator: the pools must be identical, byte for byte, and so must the renders."""
import math

import numpy as np
import pytest

import paper_1704_02724_gb300 as cx
import synth
from gpu_util import _uploaded, config_canvas, render

pytestmark = pytest.mark.gpu


def _paint_and_compare(D, E, c, r, q):
    ref = synth.stamp_canvas(D, E, c, r, q)
    _uploaded["key"] = None                      # the painter replaces the uploaded canvas
    nr, nl = cx.paint_spheres(D, E, c, r, q)
    assert (nr, nl) == (ref.n_records, ref.n_leaves)
    nodes, leaves = cx.download_octree()
    np.testing.assert_array_equal(nodes, ref.nodes)
    np.testing.assert_array_equal(leaves, ref.leaves)
    h, d = cx.octree_hash()
    assert h == d
    return ref


def test_paint_c0_identical_pools_and_image():
    D, E, c, r, q, _ = synth.config_stamps(0)
    ref = _paint_and_compare(D, E, c, r, q)
    cams = synth.config_cameras(0)
    n = synth.total_pixels(cams)
    import torch
    out = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    cx.render(cams, out)
    torch.cuda.synchronize()
    painted = out.cpu().numpy()
    img, _ = render(ref, cams, key="c0_host_painted")
    np.testing.assert_array_equal(painted, img.astype(np.float32))


@pytest.mark.parametrize("seed,D", [(1, 3), (2, 5), (3, 7), (4, 9), (5, 12), (6, 20)])
def test_paint_random_stamps(seed, D):
    """Overlapping stamps of every size: whole-canvas and outside stamps, radii down to below the finest cell,
    repeated stamps (blend order), zero extinction and zero radius."""
    rng = np.random.default_rng(seed)
    E = [1.0, 3.0, 1000.0, 40000.0][seed % 4]
    n = 300
    c = rng.uniform(-0.6, 0.6, (n, 3)) * E
    r = E * np.exp(rng.uniform(math.log(2.0 ** -(D + 1)), math.log(0.7), n))
    q = np.c_[rng.uniform(0, 1, (n, 3)), rng.uniform(0, 30, n)].astype(np.float32)
    c[:20] = c[20:40]                      # the same spheres again, other colours
    r[:20] = r[20:40]
    q[5, 3] = 0.0
    r[6] = 0.0
    c[7] = (0.0, 0.0, 0.0)
    r[7] = 2.0 * E                         # covers the whole canvas
    c[8] = (5.0 * E, 0.0, 0.0)             # outside
    _paint_and_compare(D, E, c, r, q)


def test_paint_long_lists_near_the_root():
    """More than 8192 stamps in the root's list, so the top levels take the chunked per-child passes: lists cut
    into chunks of 2048, a child painted whole by stamps spread through the order that stays a leaf (the in-order
    blend), a whole-canvas stamp halfway through, children with few or no stamps; then an append of stamps into the
    painted octant, which refines it."""
    rng = np.random.default_rng(17)
    D, E = 10, 1000.0
    n_small = 15000
    cs = rng.uniform(-0.5, -0.25, (n_small, 3)) * E            # small stamps in one corner of one octant
    rs = E * np.exp(rng.uniform(math.log(2.0 ** -11), math.log(0.02), n_small))
    cb = np.tile([0.25 * E, 0.25 * E, 0.25 * E], (30, 1))
    rb = np.full(30, 0.45 * E)                                    # each covers the whole octant x, y, z > 0
    c = np.concatenate([cs, cb])
    r = np.concatenate([rs, rb])
    order = rng.permutation(len(r))
    c, r = c[order], r[order]
    q = np.c_[rng.uniform(0, 1, (len(r), 3)), rng.uniform(0, 30, len(r))].astype(np.float32)
    mid = len(r) // 2
    c[mid] = (0.0, 0.0, 0.0)
    r[mid] = 2.0 * E                                              # the whole canvas
    _paint_and_compare(D, E, c, r, q)
    ca = rng.uniform(0.05, 0.45, (200, 3)) * E
    ra = E * np.exp(rng.uniform(math.log(2.0 ** -10), math.log(0.01), 200))
    qa = np.c_[rng.uniform(0, 1, (200, 3)), rng.uniform(0, 30, 200)].astype(np.float32)
    ref = synth.stamp_canvas(D, E, np.concatenate([c, ca]), np.concatenate([r, ra]), np.concatenate([q, qa]))
    cx.paint_append(ca, ra, qa)
    nodes, leaves = cx.download_octree()
    np.testing.assert_array_equal(nodes, ref.nodes)
    np.testing.assert_array_equal(leaves, ref.leaves)


def test_paint_empty_and_deep_reduced_c2():
    _paint_and_compare(4, 1.0, np.zeros((0, 3)), np.zeros(0), np.zeros((0, 4), np.float32))
    D, E, c, r, q, _ = synth.config_stamps(2, n_fine=4000)
    _paint_and_compare(D, E, c, r, q)


def test_paint_rejects_bad_input():
    with pytest.raises(cx.CanvoxError):
        cx.paint_spheres(8, 1.0, [[0, 0, 0]], [-1.0], [[1, 1, 1, 1]])
    with pytest.raises(cx.CanvoxError):
        cx.paint_spheres(8, 1.0, [[np.nan, 0, 0]], [0.1], [[1, 1, 1, 1]])
    with pytest.raises(cx.CanvoxError):
        cx.paint_spheres(31, 1.0, [[0, 0, 0]], [0.1], [[1, 1, 1, 1]])
    _uploaded["key"] = None


def test_paint_append_equals_whole_table():
    """Painting stamps in two calls (the second appends) gives the pools of one call over the whole table,
    the host painter's; an uploaded canvas cannot be appended to."""
    D, E, c, r, q, _ = synth.config_stamps(0)
    _uploaded["key"] = None
    cx.paint_spheres(D, E, c[:600], r[:600], q[:600])
    cx.paint_append(c[600:900], r[600:900], q[600:900])
    nr, nl = cx.paint_append(c[900:], r[900:], q[900:])
    ref = synth.build_config(0)
    assert (nr, nl) == (ref.n_records, ref.n_leaves)
    nodes, leaves = cx.download_octree()
    np.testing.assert_array_equal(nodes, ref.nodes)
    np.testing.assert_array_equal(leaves, ref.leaves)
    cx.upload_octree(ref.nodes, ref.leaves, ref.depth, ref.extent)
    with pytest.raises(cx.CanvoxError):
        cx.paint_append(c[:1], r[:1], q[:1])
    _uploaded["key"] = None


@pytest.mark.parametrize("seed,D", [(11, 3), (12, 7), (13, 12), (14, 20)])
def test_paint_append_in_chunks(seed, D):
    """Appends repaint only the partitions (refined cells of level 5) whose stamp lists change: stamps appended
    in chunks, among them one covering the whole canvas, some outside it, repeats of earlier stamps and an empty
    append, give the host painter's pools of the whole table byte for byte after every chunk."""
    rng = np.random.default_rng(seed)
    E = [1.0, 3.0, 1000.0, 40000.0][seed % 4]
    n = 400
    c = rng.uniform(-0.6, 0.6, (n, 3)) * E
    r = E * np.exp(rng.uniform(math.log(2.0 ** -(D + 1)), math.log(0.3), n))
    q = np.c_[rng.uniform(0, 1, (n, 3)), rng.uniform(0, 30, n)].astype(np.float32)
    c[300:310] = c[:10]                    # the same spheres again, later
    r[300:310] = r[:10]
    c[320] = (0.0, 0.0, 0.0)
    r[320] = 2.0 * E                       # covers the whole canvas
    c[330] = (5.0 * E, 0.0, 0.0)           # outside
    _uploaded["key"] = None
    cuts = [0, 150, 150, 290, 321, 331, 400]
    cx.paint_spheres(D, E, c[:cuts[1]], r[:cuts[1]], q[:cuts[1]])
    for a, b in zip(cuts[1:-1], cuts[2:]):
        nr, nl = cx.paint_append(c[a:b], r[a:b], q[a:b])
        ref = synth.stamp_canvas(D, E, c[:b], r[:b], q[:b])
        assert (nr, nl) == (ref.n_records, ref.n_leaves), (a, b)
        nodes, leaves = cx.download_octree()
        np.testing.assert_array_equal(nodes, ref.nodes)
        np.testing.assert_array_equal(leaves, ref.leaves)
    h, d = cx.octree_hash()
    assert h == d
    _uploaded["key"] = None


def test_paint_append_reduced_c2_localised():
    """The editing case the append is for: the last stamps of a room appended to the depth-24 canvas painted from
    the others (only the partition around that room is painted again), pools equal to the host painter's."""
    D, E, c, r, q, _ = synth.config_stamps(2, n_fine=4000)
    k = r.shape[0] - 100
    _uploaded["key"] = None
    cx.paint_spheres(D, E, c[:k], r[:k], q[:k])
    nr, nl = cx.paint_append(c[k:], r[k:], q[k:])
    ref = synth.stamp_canvas(D, E, c, r, q)
    assert (nr, nl) == (ref.n_records, ref.n_leaves)
    nodes, leaves = cx.download_octree()
    np.testing.assert_array_equal(nodes, ref.nodes)
    np.testing.assert_array_equal(leaves, ref.leaves)
    _uploaded["key"] = None


def test_paint_ties_on_cell_planes():
    """Stamps whose spheres touch cell faces, corners and centres exactly (distances equal to the radius) and whose
    radius puts r/10 exactly on a cell size: every comparison of the painter meets its tie."""
    D, E = 7, 1.0
    w = E / 2.0 ** 4
    c, r = [], []
    for i in range(-3, 4):
        for j in (-2, 0, 1):
            c.append((i * w, j * w, 0.5 * w * (i % 2)))           # on planes and cell centres
            r.append([w, 2 * w, 0.5 * w, 10 * w, 10 * E / 2.0 ** 6][(i + j) % 5])
    c = np.array(c)
    r = np.array(r)
    rng = np.random.default_rng(11)
    q = np.c_[rng.uniform(0, 1, (len(r), 3)), rng.uniform(0.5, 9.0, len(r))].astype(np.float32)
    _paint_and_compare(D, E, c, r, q)


def test_paint_depth27_million_stamps_identical_to_host():
    """The depth-27 canvas of 1,000,000 fine stamps (config 3): more than 2^31 leaves, so the pools store leaf
    numbers modulo 2^31. The device painter's pools equal the host painter's byte for byte, and the library's
    own hash of the painted pools equals the host-side hash of the host painter's pools."""
    ref = config_canvas(3)
    assert ref.n_leaves > 2 ** 31
    D, E, c, r, q, _ = synth.config_stamps(3)
    _uploaded["key"] = None
    nr, nl = cx.paint_spheres(D, E, c, r, q)
    assert (nr, nl) == (ref.n_records, ref.n_leaves)
    _, dev_hash = cx.octree_hash()
    nodes, leaves = cx.download_octree()
    assert np.array_equal(nodes, ref.nodes)
    del nodes
    assert np.array_equal(leaves, ref.leaves)
    del leaves
    cx.upload_octree(ref.nodes, ref.leaves, ref.depth, ref.extent)   # validation passes, hashes agree
    h, d = cx.octree_hash()
    assert h == d == dev_hash
    _uploaded["key"] = None
