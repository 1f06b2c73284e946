"""The seeded input generator: blend rule, stamp coverage, canonical pools, determinism (CPU)."""
import numpy as np

import synth
from bruteforce import DenseGrid


def test_splitmix64_reference_values():
    # SplitMix64 of seed 0: first outputs 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4 (Steele et al. 2014)
    r = synth.Rng(0)
    u = r.uniform(2)
    assert u[0] == (0xE220A8397B1DCDAF >> 11) / 2.0 ** 53
    assert u[1] == (0x6E789E6AA1B965F4 >> 11) / 2.0 ** 53


def test_single_stamp_paints_target_level_centres():
    """One sphere paints exactly the target-level cells whose centre lies inside it (Sec. 5.2)."""
    D = 5
    c = np.array([[0.1, -0.07, 0.2]])
    r = np.array([4.1 / 32])          # r/10 = 0.41/32 -> target depth 5 (cell 1/32)
    q = np.array([[0.25, 0.5, 0.75, 3.0]], np.float32)
    cv = synth.stamp_canvas(D, 1.0, c, r, q)
    g = DenseGrid(cv)
    N = 32
    idx = (np.arange(N) + 0.5) / N - 0.5
    X, Y, Z = np.meshgrid(idx, idx, idx, indexing="ij")
    inside = (X - c[0, 0]) ** 2 + (Y - c[0, 1]) ** 2 + (Z - c[0, 2]) ** 2 < r[0] ** 2
    assert np.array_equal(g.sigma > 0, inside)
    assert np.all(g.sigma[inside] == 3.0)
    assert np.all(g.rgb[inside] == np.array([0.25, 0.5, 0.75]))


def test_blend_of_two_stamps_closed_form():
    """Overlap colour = B m + (1 - m) C with m = B_a / (B_a + C_a), alpha = B_a + C_a (Sec. 5.1), in FP32."""
    c = np.array([[0.0, 0.0, 0.0], [0.05, 0.0, 0.0]])
    r = np.array([0.2, 0.2])
    q = np.array([[0.9, 0.1, 0.3, 2.0], [0.2, 0.6, 0.8, 6.0]], np.float32)
    cv = synth.stamp_canvas(4, 1.0, c, r, q)
    g = DenseGrid(cv)
    both = g.sigma == np.float16(np.float32(8.0))
    assert both.any()
    B, C = q[1], q[0]
    m = np.float32(B[3]) / (np.float32(B[3]) + np.float32(C[3]))
    rgb = B[0:3] * m + (np.float32(1) - m) * C[0:3]
    expect = rgb.astype(np.float32).astype(np.float16).astype(np.float64)
    assert np.all(g.rgb[both] == expect)


def test_pools_are_canonical_bfs_and_merged():
    cv = synth.build_config(0)
    nodes = cv.nodes
    internal = nodes[nodes > 0]
    assert np.array_equal(internal, np.arange(1, cv.n_records))       # each record referenced once, BFS order
    leaves = -nodes[nodes < 0] - 1
    assert np.array_equal(leaves, np.arange(cv.n_leaves))              # leaves numbered in BFS order
    lv = cv.leaves
    assert np.all(lv[:, 3] != 0)                                       # empties are slot 0, never stored
    # no record (except the root) has 8 bit-identical leaf children
    for r in range(1, min(cv.n_records, 20000)):
        s = nodes[r]
        if np.all(s <= 0):
            keys = [0 if v == 0 else lv[-v - 1].tobytes() for v in s]
            assert len(set(keys)) > 1


def test_deterministic_and_partition_exact():
    L = synth.lib()
    try:
        L.synth_set_split(1 << 30)
        L.synth_set_threads(1)
        a = synth.build_config(2, n_fine=2000)
        L.synth_set_split(64)
        L.synth_set_threads(4)
        b = synth.build_config(2, n_fine=2000)
    finally:
        L.synth_set_split(512)
        L.synth_set_threads(0)
    assert a.levels == 24
    assert np.array_equal(a.nodes, b.nodes) and np.array_equal(a.leaves, b.leaves)


def test_camera_records():
    cams = synth.config_cameras(2)
    assert cams.shape == (2,) and cams.dtype.itemsize == 136
    assert synth.total_pixels(cams) == 2 * 2160 * 2160
    eyes = cams["eye"]
    assert abs(np.linalg.norm(eyes[0] - eyes[1]) - 0.064) < 1e-12
    c3 = synth.config_cameras(3)
    assert c3.shape == (16,) and synth.total_pixels(c3) == 16 * 2160 * 2160
    c4 = synth.config_cameras(4)
    assert c4.shape == (64,)
    assert np.all((c4["width"] >= 256) & (c4["width"] <= 2160))


def test_root_array_keeps_top_levels():
    """root_levels = 2: the 4^3 array of octree roots (Sec. 4) stored as records 1-8 everywhere; the dense
    field is unchanged, and so is the image (coarsening invariance of the oracle)."""
    import math

    import oracle
    rng = synth.Rng(7)
    n = 30
    U = rng.uniform(n * 8).reshape(n, 8)
    c = np.r_[0.05 + 0.4 * U[:, 0:3], [[-0.3, -0.3, -0.3]]]
    r = np.r_[(1.0 + 6.0 * U[:, 3]) / 64.0, [2.0]]   # the last stamp paints the whole canvas first ...
    q = np.r_[np.c_[U[:, 4:7], 0.5 + 19.5 * U[:, 7]], [[0.3, 0.6, 0.9, 1.5]]].astype(np.float32)
    order = np.r_[n, np.arange(n)]                    # ... so every level-1 cell is a painted leaf or refined
    a = synth.stamp_canvas(6, 1.0, c[order], r[order], q[order])
    b = synth.stamp_canvas(6, 1.0, c[order], r[order], q[order], root_levels=2)
    assert np.all(b.nodes[0] == np.arange(1, 9))
    assert np.any(a.nodes[0] < 0)                     # merged: some octants are single leaves
    ga, gb = DenseGrid(a), DenseGrid(b)
    assert np.array_equal(ga.sigma, gb.sigma) and np.array_equal(ga.rgb, gb.rgb)
    cam = synth.cameras_array([synth.look_at_camera([1.2, 0.9, 1.7], [0, 0, 0], [0, 1, 0], math.tan(math.radians(30)),
                                                    40, 30, 0, (0.1, 0.2, 0.3, 1))])
    np.testing.assert_allclose(oracle.render(b, cam, t_min=0.0), oracle.render(a, cam, t_min=0.0), rtol=0, atol=1e-13)
