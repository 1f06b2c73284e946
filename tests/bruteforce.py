"""Brute-force uniform-grid ray marcher (test instrument that pins the oracle).

The octree is expanded to its dense finest grid (2^D cells per axis). Along a
ray every grid-plane crossing time is collected and sorted; each interval is
classified by the voxel that holds its midpoint, so no tie rules, no tree
descent and no leaf exits are involved. The emission-absorption sum is then
taken interval by interval. Amanatides and Woo (1987) march the same cells
incrementally; here all crossings are enumerated at once.
"""
import math

import numpy as np


class DenseGrid:
    def __init__(self, canvas):
        D = canvas.levels if canvas.levels else canvas.depth
        D = max(D, _tree_depth(canvas.nodes))
        self.N = N = 1 << D
        self.E = float(canvas.extent)
        self.sigma = np.zeros((N, N, N))
        self.rgb = np.zeros((N, N, N, 3))
        self.leaf = np.full((N, N, N), -1, dtype=np.int64)
        self.paths = {}
        lv = canvas.leaves.view(np.float16).astype(np.float64) if canvas.leaves.size else np.zeros((0, 4))
        # explicit stack: (record, level, x0, y0, z0, path)
        stack = [(0, 0, 0, 0, 0, ())]
        while stack:
            rec, level, x0, y0, z0, path = stack.pop()
            n = N >> (level + 1)
            for k in range(8):
                x = x0 + (k & 1) * n
                y = y0 + ((k >> 1) & 1) * n
                z = z0 + ((k >> 2) & 1) * n
                v = int(canvas.nodes[rec, k])
                p = path + (k,)
                if v > 0:
                    stack.append((v, level + 1, x, y, z, p))
                    continue
                lid = rec * 8 + k
                self.paths[lid] = p
                self.leaf[x:x + n, y:y + n, z:z + n] = lid
                if v < 0:
                    q = lv[-v - 1]
                    self.sigma[x:x + n, y:y + n, z:z + n] = q[3]
                    self.rgb[x:x + n, y:y + n, z:z + n] = q[0:3]


def _tree_depth(nodes):
    depth = np.zeros(nodes.shape[0], dtype=np.int64)
    for r in range(nodes.shape[0]):
        for v in nodes[r]:
            if v > 0:
                depth[v] = depth[r] + 1
    return int(depth.max()) + 1


def march(grid, o, d, bg=(0.0, 0.0, 0.0, 0.0), t_min=0.0, visited=None):
    """Returns (rgba, steps, reads): steps = leaves entered, reads = slot reads with a perfect stack.
    With a list `visited`, appends the id (record * 8 + child) of every leaf entered."""
    o = [float(x) for x in o]
    bg = [float(x) for x in np.asarray(bg, dtype=np.float32)]  # the camera record stores FP32 background
    d = np.asarray(d, dtype=np.float64)
    d = d / math.sqrt(float(d @ d))
    d = [float(x) for x in d]
    h = 0.5 * grid.E
    w = grid.E / grid.N
    t0, t1 = 0.0, math.inf
    for a in range(3):
        if d[a] != 0.0:
            ta, tb = (-h - o[a]) / d[a], (h - o[a]) / d[a]
            t0 = max(t0, min(ta, tb))
            t1 = min(t1, max(ta, tb))
        elif not (-h <= o[a] < h):
            t1 = -math.inf
    C = [0.0, 0.0, 0.0]
    T = 1.0
    steps = reads = 0
    if t0 < t1:
        ts = {t0, t1}
        for a in range(3):
            if d[a] == 0.0:
                continue
            for i in range(grid.N + 1):
                t = (-h + i * w - o[a]) / d[a]
                if t0 < t < t1:
                    ts.add(t)
        ts = sorted(ts)
        prev_leaf, prev_path = None, None
        for ta, tb in zip(ts[:-1], ts[1:]):
            tm = 0.5 * (ta + tb)
            idx = [min(grid.N - 1, max(0, int(math.floor((o[a] + tm * d[a] + h) / w)))) for a in range(3)]
            lid = int(grid.leaf[idx[0], idx[1], idx[2]])
            if lid != prev_leaf:
                if visited is not None:
                    visited.append(lid)
                p = grid.paths[lid]
                common = 0
                if prev_path is not None:
                    while common < min(len(p), len(prev_path)) and p[common] == prev_path[common]:
                        common += 1
                reads += len(p) - common
                steps += 1
                prev_leaf, prev_path = lid, p
            s = float(grid.sigma[idx[0], idx[1], idx[2]])
            if s > 0.0:
                l = tb - ta
                a_ = -math.expm1(-s * l)
                c = grid.rgb[idx[0], idx[1], idx[2]]
                for ch in range(3):
                    C[ch] += T * a_ * float(c[ch])
                T *= math.exp(-s * l)
            if T < t_min:
                break
    return np.array([C[0] + T * bg[0], C[1] + T * bg[1], C[2] + T * bg[2], 1.0 - T]), steps, reads
