"""GB300 (sm_103a) ray caster for deep sparse octree canvases.

The renderer of CanvoX (arXiv 1704.02724, Sec. 6): one ray per pixel through
an octree of depth up to 30, front-to-back emission-absorption compositing,
early termination at full opacity. The work runs in ``libcanvox.so`` (CUDA
kernels behind the C ABI of ``include/canvox.h``); ``canvox`` is a thin
ctypes binding with the same entry points.
"""
from .canvox import (  # noqa: F401
    CanvoxError,
    PREC_MIXED,
    PREC_FP64,
    PREC_FP32,
    PREC_CELL32,
    PREC_WORLD32,
    PREC_CELL16,
    PREC_FP64_LINKS,
    lib,
    upload_octree,
    render,
    render_host,
    render_noalloc,
    get_stats,
    octree_hash,
    autotune,
    footprint,
    paint_spheres,
    paint_append,
    canvas_info,
    update_leaves,
    download_octree,
    probe_l2_gather,
    probe_fp64,
    default_opts,
    last_error,
    release,
)
