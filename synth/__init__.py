"""Seeded synthetic inputs for the deep-octree renderer: canvases and cameras.

This module is the only code that both the CUDA path and the FP64 oracle use.
It produces inputs (octree pools, camera records); it holds none of the
ray-casting arithmetic.

Canvases are built by stamping spheres into an adaptive octree (Sec. 5.1-5.2
of the paper: additive blend, about ten cells per brush radius, conservative
coarsening), quantised to FP16 and laid out breadth-first (Sec. 4.1.1).
The five workloads are listed in ``synth.configs``.
"""
import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

from . import _build

# Camera record, 136 bytes, little-endian, no padding. Both renderers take an
# array of these: eye/right/up/forward in canvas coordinates (FP64), tangent of
# half the vertical field of view, image size, first pixel of the view in the
# output image, and the background RGBA.
CAM_DTYPE = np.dtype([
    ("eye", "<f8", (3,)),
    ("right", "<f8", (3,)),
    ("up", "<f8", (3,)),
    ("forward", "<f8", (3,)),
    ("tan_half_fov_y", "<f8"),
    ("width", "<i4"),
    ("height", "<i4"),
    ("out_offset_px", "<i8"),
    ("background", "<f4", (4,)),
])
assert CAM_DTYPE.itemsize == 136

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.synth_splitmix_uniform.argtypes = [ctypes.POINTER(ctypes.c_uint64), ctypes.c_int64, ctypes.c_void_p]
        L.synth_splitmix_uniform.restype = None
        L.synth_log_uniform.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
        L.synth_log_uniform.restype = None
        L.synth_tree_new.argtypes = [ctypes.c_int32, ctypes.c_double]
        L.synth_tree_new.restype = ctypes.c_void_p
        L.synth_tree_free.argtypes = [ctypes.c_void_p]
        L.synth_tree_free.restype = None
        L.synth_tree_stamp_spheres.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.synth_tree_stamp_spheres.restype = ctypes.c_int
        L.synth_tree_finalize.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)]
        L.synth_tree_finalize.restype = ctypes.c_int
        L.synth_tree_export.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.synth_tree_export.restype = ctypes.c_int
        L.synth_tree_sizes.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
        L.synth_tree_sizes.restype = None
        L.synth_tree_set_root_levels.argtypes = [ctypes.c_void_p, ctypes.c_int32]
        L.synth_tree_set_root_levels.restype = ctypes.c_int
        L.synth_set_threads.argtypes = [ctypes.c_int32]
        L.synth_set_threads.restype = None
        L.synth_set_split.argtypes = [ctypes.c_int32]
        L.synth_set_split.restype = None
        _lib = L
    return _lib


class Rng:
    """SplitMix64 stream of uniform doubles in [0, 1) (top 53 bits)."""

    def __init__(self, seed):
        self.state = ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF)

    def uniform(self, n):
        out = np.empty(int(n), dtype=np.float64)
        lib().synth_splitmix_uniform(ctypes.byref(self.state), int(n), out.ctypes.data)
        return out


def log_uniform(a, b, u):
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.empty_like(u)
    lib().synth_log_uniform(float(a), float(b), u.ctypes.data, u.size, out.ctypes.data)
    return out


@dataclass
class Canvas:
    """Canonical pools: nodes int32[n_rec, 8], leaves uint16[n_leaf, 4] (FP16 bits R,G,B,sigma)."""
    nodes: np.ndarray
    leaves: np.ndarray
    depth: int
    extent: float
    levels: int = 0
    info: dict = field(default_factory=dict)

    @property
    def n_records(self):
        return int(self.nodes.shape[0])

    @property
    def n_leaves(self):
        return int(self.leaves.shape[0])


def stamp_canvas(depth, extent, centers, radii, rgba, root_levels=1):
    """Build a canvas from spherical stamps applied in order. root_levels = 2 keeps the top two
    levels refined everywhere: the 4^3 array of octree roots (the level-2 cells) of Sec. 4."""
    L = lib()
    centers = np.ascontiguousarray(centers, dtype=np.float64).reshape(-1, 3)
    radii = np.ascontiguousarray(radii, dtype=np.float64).reshape(-1)
    rgba = np.ascontiguousarray(rgba, dtype=np.float32).reshape(-1, 4)
    n = radii.shape[0]
    assert centers.shape[0] == n and rgba.shape[0] == n
    h = L.synth_tree_new(int(depth), float(extent))
    if not h:
        raise ValueError("bad depth/extent")
    try:
        if root_levels != 1 and L.synth_tree_set_root_levels(h, int(root_levels)) != 0:
            raise ValueError("root_levels must be in [1, depth)")
        if n:
            rc = L.synth_tree_stamp_spheres(h, n, centers.ctypes.data, radii.ctypes.data, rgba.ctypes.data)
            if rc != 0:
                raise MemoryError("more than 2^31 - 1 stamps")
        nb, nv = ctypes.c_int64(), ctypes.c_int64()
        L.synth_tree_sizes(h, ctypes.byref(nb), ctypes.byref(nv))
        nr, nl, ml = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        if L.synth_tree_finalize(h, ctypes.byref(nr), ctypes.byref(nl), ctypes.byref(ml)) != 0:
            raise MemoryError("pools beyond 2^31 - 1 records or 2^34 leaves")
        nodes = np.empty((nr.value, 8), dtype=np.int32)
        leaves = np.empty((nl.value, 4), dtype=np.uint16)
        L.synth_tree_export(h, nodes.ctypes.data, leaves.ctypes.data)
    finally:
        L.synth_tree_free(h)
    return Canvas(nodes=nodes, leaves=leaves, depth=int(depth), extent=float(extent), levels=int(ml.value),
                  info={"stamps": int(n), "build_records": int(nb.value), "build_values": int(nv.value)})


def look_at_camera(eye, target, up_hint, tan_half_fov_y, width, height, offset=0, background=(0, 0, 0, 0)):
    """One camera record looking from eye at target (orthonormal right/up/forward)."""
    eye = np.asarray(eye, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - eye
    f = f / np.linalg.norm(f)
    r = np.cross(f, np.asarray(up_hint, dtype=np.float64))
    r = r / np.linalg.norm(r)
    u = np.cross(r, f)
    return camera(eye, r, u, f, tan_half_fov_y, width, height, offset, background)


def camera(eye, right, up, forward, tan_half_fov_y, width, height, offset=0, background=(0, 0, 0, 0)):
    c = np.zeros((), dtype=CAM_DTYPE)
    c["eye"] = eye
    c["right"] = right
    c["up"] = up
    c["forward"] = forward
    c["tan_half_fov_y"] = tan_half_fov_y
    c["width"] = width
    c["height"] = height
    c["out_offset_px"] = offset
    c["background"] = background
    return c


def cameras_array(cams):
    """Stack camera records into a contiguous CAM_DTYPE array."""
    out = np.zeros(len(cams), dtype=CAM_DTYPE)
    for i, c in enumerate(cams):
        out[i] = c
    return out


def total_pixels(cams):
    cams = np.asarray(cams, dtype=CAM_DTYPE).reshape(-1)
    if cams.size == 0:
        return 0
    return int(np.max(cams["out_offset_px"] + cams["width"].astype(np.int64) * cams["height"].astype(np.int64)))


from .configs import CONFIGS, build_config, config_cameras, config_stamps  # noqa: E402,F401
