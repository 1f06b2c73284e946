"""FP64 CPU oracle for deep-octree ray casting. TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference legs may import this package. The product renderer
(``paper_1704_02724_gb300``) never imports it, and the two share no code:
the oracle is plain C (``oracle.c``) written from the paper's definitions
(Sec. 6: rays from an FP64 eye, leaf-by-leaf traversal to full opacity or the
canvas exit; Sec. 4.1.1: index pools, eight children per unit), evaluated in
FP64 with point location from the root at every step.

Parity of the oracle is pinned by ``tests/test_oracle_pins.py`` against a
brute-force uniform-grid ray marcher, closed forms and invariants.
"""
import ctypes

import numpy as np

from . import _build

_lib = None

T_MIN_DEFAULT = 2.0 ** -20


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(_build.build())
        L.oracle_leaf_base.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
        L.oracle_leaf_base.restype = None
        L.oracle_render.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_double,
                                    ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64,
                                    ctypes.c_double, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_int32]
        L.oracle_render.restype = ctypes.c_int64
        L.oracle_trace_rays.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_double,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                        ctypes.c_double, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p]
        L.oracle_trace_rays.restype = ctypes.c_int64
        L.oracle_footprint.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_double,
                                       ctypes.c_void_p, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]
        L.oracle_footprint.restype = ctypes.c_int64
        L.oracle_walk32.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p, ctypes.c_int32,
                                    ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]
        L.oracle_walk32.restype = ctypes.c_int64
        L.oracle_max_threads.argtypes = []
        L.oracle_max_threads.restype = ctypes.c_int32
        _lib = L
    return _lib


def max_threads():
    return int(lib().oracle_max_threads())


def _pools(canvas):
    """(nodes, leaves, leaf_base): the pools as C arrays and, per record, the number of leaf slots in the
    records before it (the oracle's leaf numbering; cached on the canvas object when it allows it)."""
    nodes = np.ascontiguousarray(canvas.nodes, dtype=np.int32)
    leaves = np.ascontiguousarray(canvas.leaves, dtype=np.uint16)
    if leaves.size == 0:
        leaves = np.zeros((1, 4), dtype=np.uint16)
    base = getattr(canvas, "_oracle_leaf_base", None)
    if base is None or base.shape[0] != nodes.shape[0]:
        base = np.empty(max(nodes.shape[0], 1), dtype=np.int64)
        lib().oracle_leaf_base(nodes.ctypes.data, nodes.shape[0], base.ctypes.data)
        try:
            canvas._oracle_leaf_base = base
        except AttributeError:
            pass
    return nodes, leaves, base


def render(canvas, cams, px_idx=None, t_min=T_MIN_DEFAULT, threads=0, counters=False, max_steps=0):
    """Render the given output pixels (all when px_idx is None) in FP64.

    Returns rgba float64 [n, 4]; with counters=True also (icount int64 [n, 3] =
    steps, slot reads from the LCA, leaf loads; dcount float64 [n, 2] = sum of
    crossed cell widths, ray length in the canvas).
    """
    nodes, leaves, base = _pools(canvas)
    cams = np.ascontiguousarray(cams)
    assert cams.dtype.itemsize == 136
    n_views = cams.shape[0]
    if px_idx is None:
        n = 0
        for c in cams:
            n = max(n, int(c["out_offset_px"]) + int(c["width"]) * int(c["height"]))
        idx_ptr = None
    else:
        px_idx = np.ascontiguousarray(px_idx, dtype=np.int64)
        n = px_idx.shape[0]
        idx_ptr = px_idx.ctypes.data
    out = np.empty((n, 4), dtype=np.float64)
    ic = np.zeros((n, 3), dtype=np.int64) if counters else None
    dc = np.zeros((n, 2), dtype=np.float64) if counters else None
    rc = lib().oracle_render(nodes.ctypes.data, leaves.ctypes.data, base.ctypes.data, int(canvas.depth),
                             float(canvas.extent),
                             cams.ctypes.data if n_views else None, int(n_views), idx_ptr, int(n),
                             float(t_min), int(max_steps), out.ctypes.data,
                             ic.ctypes.data if counters else None, dc.ctypes.data if counters else None,
                             int(threads))
    if rc != 0:
        raise RuntimeError(f"oracle_render returned {rc}")
    return (out, ic, dc) if counters else out


def trace_rays(canvas, origins, directions, background=(0, 0, 0, 0), t_min=T_MIN_DEFAULT, counters=False,
               max_steps=0):
    """Trace explicit rays (directions are normalised in FP64)."""
    nodes, leaves, base = _pools(canvas)
    o = np.ascontiguousarray(origins, dtype=np.float64).reshape(-1, 3)
    d = np.ascontiguousarray(directions, dtype=np.float64).reshape(-1, 3)
    bg = np.ascontiguousarray(background, dtype=np.float32)
    n = o.shape[0]
    out = np.empty((n, 4), dtype=np.float64)
    ic = np.zeros((n, 3), dtype=np.int64)
    dc = np.zeros((n, 2), dtype=np.float64)
    rc = lib().oracle_trace_rays(nodes.ctypes.data, leaves.ctypes.data, base.ctypes.data, int(canvas.depth),
                                 float(canvas.extent),
                                 o.ctypes.data, d.ctypes.data, n, bg.ctypes.data, float(t_min), int(max_steps),
                                 out.ctypes.data, ic.ctypes.data, dc.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"oracle_trace_rays returned {rc}")
    return (out, ic, dc) if counters else out


def footprint(canvas, cams, t_min=T_MIN_DEFAULT, threads=0):
    """Records and stored leaves the traversal reads for every pixel of these views.

    Returns (rec_mark bool [n_records], leaf_mark bool [n_leaves], rgba [n_pixels, 4]).
    """
    nodes, leaves, base = _pools(canvas)
    cams = np.ascontiguousarray(cams)
    n_views = cams.shape[0]
    n = 0
    for c in cams:
        n = max(n, int(c["out_offset_px"]) + int(c["width"]) * int(c["height"]))
    out = np.empty((max(n, 1), 4), dtype=np.float64)
    rm = np.zeros(max(nodes.shape[0], 1), dtype=np.uint8)
    lm = np.zeros(max(leaves.shape[0], 1), dtype=np.uint8)
    rc = lib().oracle_footprint(nodes.ctypes.data, leaves.ctypes.data, base.ctypes.data, int(canvas.depth),
                                float(canvas.extent),
                                cams.ctypes.data if n_views else None, int(n_views), float(t_min), out.ctypes.data,
                                rm.ctypes.data, lm.ctypes.data, int(threads))
    if rc != 0:
        raise RuntimeError(f"oracle_footprint returned {rc}")
    return rm[:nodes.shape[0]].astype(bool), lm[:canvas.n_leaves].astype(bool), out[:n]


def walk32(canvas, cams, cell_local=True, threads=0, max_steps=0):
    """The paper's FP32 walk (cell-local, or in canvas coordinates) to the canvas exit, geometry only.

    Returns (steps int32 [n_pixels], angle_deg float64 [n_pixels]); pixels of no view: -1, NaN.
    """
    nodes = np.ascontiguousarray(canvas.nodes, dtype=np.int32)
    cams = np.ascontiguousarray(cams)
    n = 0
    for c in cams:
        n = max(n, int(c["out_offset_px"]) + int(c["width"]) * int(c["height"]))
    steps = np.empty(max(n, 1), dtype=np.int32)
    angle = np.empty(max(n, 1), dtype=np.float64)
    rc = lib().oracle_walk32(nodes.ctypes.data, int(canvas.depth), float(canvas.extent),
                             cams.ctypes.data if cams.shape[0] else None, int(cams.shape[0]), int(bool(cell_local)),
                             int(max_steps), steps.ctypes.data, angle.ctypes.data, int(threads))
    if rc != 0:
        raise RuntimeError(f"oracle_walk32 returned {rc}")
    return steps[:n], angle[:n]
