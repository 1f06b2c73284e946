"""Seeded random octrees with arbitrary refinement (inputs for pins and edge cases).

Unlike the stamp canvases, these trees put leaves of very different levels
side by side, include empty leaves anywhere, and can be left un-merged.
"""
import numpy as np

from . import Canvas, Rng


def _half_bits(x):
    return np.asarray(x, dtype=np.float16).view(np.uint16)


def from_nested(tree, depth, extent):
    """Breadth-first pools from a nested description.

    ``tree`` is a list of 8 entries (child k = x + 2y + 4z); an entry is either a
    list of 8 (an internal cell), None (empty leaf) or a tuple (r, g, b, sigma).
    """
    nodes, leaves = [], []
    queue = [tree]
    next_rec = 1
    qi = 0
    while qi < len(queue):
        cell = queue[qi]
        qi += 1
        rec = []
        for child in cell:
            if isinstance(child, list):
                rec.append(next_rec)
                next_rec += 1
                queue.append(child)
            elif child is None:
                rec.append(0)
            else:
                leaves.append(child)
                rec.append(-len(leaves))
        nodes.append(rec)
    nodes = np.array(nodes, dtype=np.int32).reshape(-1, 8)
    lv = _half_bits(np.array(leaves, dtype=np.float64).reshape(-1, 4)) if leaves else np.zeros((0, 4), np.uint16)
    return Canvas(nodes=nodes, leaves=np.ascontiguousarray(lv), depth=int(depth), extent=float(extent))


def random_nested(depth, seed, p_refine=0.45, p_empty=0.3, sigma_range=(0.5, 20.0), min_level=1):
    """Random refinement: each cell below depth splits with probability p_refine
    (always above min_level); leaves are empty with probability p_empty."""
    rng = Rng(seed)

    def cell(level):
        out = []
        for _ in range(8):
            u = rng.uniform(6)
            if level + 1 < depth and (level + 1 < min_level or u[0] < p_refine):
                out.append(cell(level + 1))
            elif u[1] < p_empty:
                out.append(None)
            else:
                s = sigma_range[0] + (sigma_range[1] - sigma_range[0]) * u[5]
                out.append((u[2], u[3], u[4], s))
        return out

    return cell(0)


def random_tree(depth, seed, extent=1.0, **kw):
    return from_nested(random_nested(depth, seed, **kw), depth, extent)


def uniform_tree(depth, value, extent=1.0):
    """Every cell refined down to ``depth`` with the same leaf value (not merged)."""
    def cell(level):
        if level + 1 < depth:
            return [cell(level + 1) for _ in range(8)]
        return [value] * 8
    return from_nested(cell(0), depth, extent)


def mirror_x(tree):
    """Reflect a nested tree across the x = 0 plane (child bit x flipped at every level)."""
    if not isinstance(tree, list):
        return tree
    return [mirror_x(tree[k ^ 1]) for k in range(8)]


def embed(tree, small_depth, level, cell_index):
    """Place a nested tree as the cell ``cell_index`` (ix, iy, iz) at ``level``; everything else empty."""
    node = tree
    for l in range(level, 0, -1):
        # the ancestor at level l-1 has this node as child k, k from bit (level - l) of the indices
        b = level - l
        k = ((cell_index[0] >> b) & 1) | (((cell_index[1] >> b) & 1) << 1) | (((cell_index[2] >> b) & 1) << 2)
        parent = [None] * 8
        parent[k] = node
        node = parent
    return node


def nested_depth(tree):
    if not isinstance(tree, list):
        return 0
    return 1 + max(nested_depth(c) for c in tree)
