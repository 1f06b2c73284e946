"""ctypes binding of libcanvox.so (include/canvox.h): argument marshalling only.

Every step of rendering runs in the library's CUDA kernels. PyTorch is used,
when present, only to obtain device pointers and the current CUDA stream.
The library must have been built (``paper_1704_02724_gb300._build.build()``
or ``__graft_entry__.build()``); there is no fallback path.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcanvox.so")   # the library build() makes, nothing else

OK = 0
ERR_INVALID_ARG = -1
ERR_NOT_UPLOADED = -2
ERR_BAD_TREE = -3
ERR_CUDA = -4
ERR_OOM = -5
ERR_STEP_LIMIT = -6
ERR_NAMES = {-1: "INVALID_ARG", -2: "NOT_UPLOADED", -3: "BAD_TREE", -4: "CUDA", -5: "OOM", -6: "STEP_LIMIT"}

PREC_MIXED = 0
PREC_FP64 = 1
PREC_FP32 = 2
PREC_CELL32 = 3
PREC_WORLD32 = 4
PREC_CELL16 = 5
PREC_FP64_LINKS = 6

# canvox_camera: 136 bytes (eye, right, up, forward: FP64[3]; tan; width, height; offset; background FP32[4])
CAMERA_BYTES = 136


class CanvoxError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"canvox error {code} ({ERR_NAMES.get(code, '?')}): {msg}")
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int32),
        ("per_view", ctypes.c_int32),
        ("use_graph", ctypes.c_int32),
        ("block_threads", ctypes.c_int32),
        ("blocks_per_sm", ctypes.c_int32),
        ("refill", ctypes.c_int32),
        ("smem_records", ctypes.c_int32),
        ("frame_levels", ctypes.c_int32),
        ("tile_w", ctypes.c_int32),
        ("traversal", ctypes.c_int32),
        ("step_limit", ctypes.c_int64),
        ("t_min", ctypes.c_float),
        ("err_budget", ctypes.c_float),
        ("step_count", ctypes.c_void_p),
        ("angle_deg", ctypes.c_void_p),
        ("count_reads", ctypes.c_int32),
    ]


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "rays", "steps", "slot_reads", "leaf_loads", "record_loads", "fp64_boundaries", "rebases", "step_limited",
        "h2d_bytes", "d2h_bytes")]


_lib = None


def lib():
    """Load libcanvox.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1704_02724_gb300._build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        L.canvox_default_opts.argtypes = [ctypes.POINTER(Opts)]
        L.canvox_default_opts.restype = None
        L.canvox_upload_octree.argtypes = [vp, i64, vp, i64, i32, ctypes.c_double]
        L.canvox_upload_octree.restype = ctypes.c_int
        L.canvox_render.argtypes = [vp, i32, vp, vp]
        L.canvox_render.restype = ctypes.c_int
        L.canvox_render_ex.argtypes = [vp, i32, vp, vp, ctypes.POINTER(Opts)]
        L.canvox_render_ex.restype = ctypes.c_int
        L.canvox_render_host.argtypes = [vp, i32, vp, vp, ctypes.POINTER(Opts)]
        L.canvox_render_host.restype = ctypes.c_int
        L.canvox_render_noalloc.argtypes = [vp, i64, vp, i64, i32, ctypes.c_double, vp, i32, vp, vp]
        L.canvox_render_noalloc.restype = ctypes.c_int
        L.canvox_get_stats.argtypes = [ctypes.POINTER(Stats)]
        L.canvox_get_stats.restype = ctypes.c_int
        L.canvox_octree_hash.argtypes = [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]
        L.canvox_octree_hash.restype = ctypes.c_int
        L.canvox_autotune.argtypes = [vp, i32, vp, ctypes.POINTER(Opts)]
        L.canvox_autotune.restype = ctypes.c_int
        L.canvox_footprint.argtypes = [vp, i32, vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
        L.canvox_footprint.restype = ctypes.c_int
        L.canvox_probe_l2_gather.argtypes = [i64, ctypes.POINTER(ctypes.c_double)]
        L.canvox_probe_l2_gather.restype = ctypes.c_int
        L.canvox_probe_fp64.argtypes = [ctypes.POINTER(ctypes.c_double)]
        L.canvox_probe_fp64.restype = ctypes.c_int
        L.canvox_paint_spheres.argtypes = [i32, ctypes.c_double, vp, vp, vp, i64, ctypes.POINTER(ctypes.c_int64),
                                           ctypes.POINTER(ctypes.c_int64)]
        L.canvox_paint_spheres.restype = ctypes.c_int
        L.canvox_paint_append.argtypes = [vp, vp, vp, i64, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
        L.canvox_paint_append.restype = ctypes.c_int
        L.canvox_update_leaves.argtypes = [i64, i64, vp]
        L.canvox_update_leaves.restype = ctypes.c_int
        L.canvox_canvas_info.argtypes = [ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                         ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)]
        L.canvox_canvas_info.restype = ctypes.c_int
        L.canvox_download_octree.argtypes = [vp, vp]
        L.canvox_download_octree.restype = ctypes.c_int
        L.canvox_last_error.argtypes = []
        L.canvox_last_error.restype = ctypes.c_char_p
        L.canvox_release.argtypes = []
        L.canvox_release.restype = None
        _lib = L
    return _lib


def last_error():
    return lib().canvox_last_error().decode()


def _check(rc):
    if rc != OK:
        raise CanvoxError(rc, last_error())


def _opts_to_dict(o):
    return {n: getattr(o, n) for n, _ in Opts._fields_ if n not in ("step_count", "angle_deg")}


def default_opts():
    o = Opts()
    lib().canvox_default_opts(ctypes.byref(o))
    return _opts_to_dict(o)


def make_opts(**kw):
    o = Opts()
    lib().canvox_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if k in ("step_count", "angle_deg"):
            v = _dev_ptr(v) if v is not None else None
        elif not hasattr(o, k):
            raise TypeError(f"unknown render option {k!r}")
        setattr(o, k, v)
    return o


def _cams(cams):
    cams = np.ascontiguousarray(cams)
    if cams.dtype.itemsize != CAMERA_BYTES:
        raise TypeError("cameras must be an array of 136-byte canvox_camera records")
    return cams


def _dev_ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def upload_octree(nodes, leaves, depth, extent):
    """Validate and copy the pools to the current device (see canvox_upload_octree)."""
    nodes = np.ascontiguousarray(nodes, dtype=np.int32).reshape(-1, 8)
    leaves = np.ascontiguousarray(leaves, dtype=np.uint16).reshape(-1, 4)
    _check(lib().canvox_upload_octree(nodes.ctypes.data, nodes.shape[0],
                                      leaves.ctypes.data if leaves.size else None, leaves.shape[0],
                                      int(depth), float(extent)))


def render(cams, out, stream=None, **opts):
    """Render views into a device float32 RGBA buffer (torch tensor or device pointer); asynchronous."""
    cams = _cams(cams)
    o = make_opts(**opts)
    _check(lib().canvox_render_ex(cams.ctypes.data if cams.size else None, cams.shape[0], _dev_ptr(out),
                                  _stream_ptr(stream), ctypes.byref(o)))


def render_host(cams, out, stream=None, **opts):
    """Render into a host float32 array [n_pixels, 4] (pinned copies fastest); synchronous."""
    cams = _cams(cams)
    o = make_opts(**opts)
    if isinstance(out, np.ndarray):
        if out.dtype != np.float32 or not out.flags["C_CONTIGUOUS"]:
            raise TypeError("out must be a C-contiguous float32 array")
        ptr = out.ctypes.data
    else:
        ptr = int(out.data_ptr())
    _check(lib().canvox_render_host(cams.ctypes.data if cams.size else None, cams.shape[0], ptr,
                                    _stream_ptr(stream), ctypes.byref(o)))


def render_noalloc(nodes_dev, n_records, leaves_dev, n_leaves, depth, extent, cams, out, stream=None):
    """canvox_render_noalloc: caller-owned device pools and image, no allocation by the library."""
    cams = _cams(cams)
    _check(lib().canvox_render_noalloc(_dev_ptr(nodes_dev), int(n_records), _dev_ptr(leaves_dev), int(n_leaves),
                                       int(depth), float(extent), cams.ctypes.data if cams.size else None,
                                       cams.shape[0], _dev_ptr(out), _stream_ptr(stream)))


def get_stats(check=True):
    s = Stats()
    rc = lib().canvox_get_stats(ctypes.byref(s))
    d = {n: getattr(s, n) for n, _ in Stats._fields_}
    if check and rc != ERR_STEP_LIMIT:
        _check(rc)
    d["status"] = rc
    return d


def octree_hash():
    h, d = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().canvox_octree_hash(ctypes.byref(h), ctypes.byref(d)))
    return h.value, d.value


def autotune(cams, stream=None):
    cams = _cams(cams)
    o = Opts()
    _check(lib().canvox_autotune(cams.ctypes.data, cams.shape[0], _stream_ptr(stream), ctypes.byref(o)))
    return _opts_to_dict(o)


def paint_spheres(depth, extent, centers, radii, rgba):
    """canvox_paint_spheres: build the canvas of these stamps on the GPU; returns (n_records, n_leaves)."""
    c = np.ascontiguousarray(centers, dtype=np.float64).reshape(-1, 3)
    r = np.ascontiguousarray(radii, dtype=np.float64).reshape(-1)
    q = np.ascontiguousarray(rgba, dtype=np.float32).reshape(-1, 4)
    n = r.shape[0]
    if c.shape[0] != n or q.shape[0] != n:
        raise ValueError("centers, radii and rgba must have one row per stamp")
    nr, nl = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().canvox_paint_spheres(int(depth), float(extent), c.ctypes.data if n else None,
                                      r.ctypes.data if n else None, q.ctypes.data if n else None, n,
                                      ctypes.byref(nr), ctypes.byref(nl)))
    return nr.value, nl.value


def paint_append(centers, radii, rgba):
    """canvox_paint_append: add stamps to the painted canvas and repaint; returns (n_records, n_leaves)."""
    c = np.ascontiguousarray(centers, dtype=np.float64).reshape(-1, 3)
    r = np.ascontiguousarray(radii, dtype=np.float64).reshape(-1)
    q = np.ascontiguousarray(rgba, dtype=np.float32).reshape(-1, 4)
    n = r.shape[0]
    if c.shape[0] != n or q.shape[0] != n:
        raise ValueError("centers, radii and rgba must have one row per stamp")
    nr, nl = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().canvox_paint_append(c.ctypes.data if n else None, r.ctypes.data if n else None,
                                     q.ctypes.data if n else None, n, ctypes.byref(nr), ctypes.byref(nl)))
    return nr.value, nl.value


def update_leaves(first, leaf_rgba):
    """canvox_update_leaves: new values for leaves [first, first + len(leaf_rgba)) of the current canvas."""
    q = np.ascontiguousarray(leaf_rgba, dtype=np.uint16).reshape(-1, 4)
    _check(lib().canvox_update_leaves(int(first), q.shape[0], q.ctypes.data if q.size else None))


def canvas_info():
    """canvox_canvas_info: (n_records, n_leaves, depth, extent) of the current canvas."""
    nr, nl, d, e = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_double()
    _check(lib().canvox_canvas_info(ctypes.byref(nr), ctypes.byref(nl), ctypes.byref(d), ctypes.byref(e)))
    return nr.value, nl.value, d.value, e.value


def download_octree():
    """canvox_download_octree: (node_pool int32 [n_records, 8], leaf_rgba uint16 [n_leaves, 4])."""
    nr, nl, _, _ = canvas_info()
    nodes = np.empty((nr, 8), dtype=np.int32)
    leaves = np.empty((max(nl, 1), 4), dtype=np.uint16)
    _check(lib().canvox_download_octree(nodes.ctypes.data, leaves.ctypes.data))
    return nodes, leaves[:nl]


def footprint(cams, stream=None):
    """canvox_footprint: (distinct records, distinct stored leaves) the rays of these views read."""
    cams = _cams(cams)
    r, l_ = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().canvox_footprint(cams.ctypes.data if cams.size else None, cams.shape[0], _stream_ptr(stream),
                                  ctypes.byref(r), ctypes.byref(l_)))
    return r.value, l_.value


def probe_l2_gather(buffer_bytes=0):
    """canvox_probe_l2_gather: GB/s of random 32-byte sector gathers served by L2."""
    v = ctypes.c_double()
    _check(lib().canvox_probe_l2_gather(int(buffer_bytes), ctypes.byref(v)))
    return v.value


def probe_fp64():
    """canvox_probe_fp64: FP64 FMA GFLOP/s."""
    v = ctypes.c_double()
    _check(lib().canvox_probe_fp64(ctypes.byref(v)))
    return v.value


def release():
    lib().canvox_release()
