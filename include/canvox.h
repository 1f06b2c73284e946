/*
 * canvox.h - C ABI of the GB300 deep-octree ray caster (libcanvox.so).
 *
 * The library renders a canvas stored as a deep sparse octree (depth 1..30)
 * by casting one ray per pixel, compositing the leaves' colour and extinction
 * front to back and stopping early at full opacity (the rendering problem of
 * Sec. 6 of "CanvoX: High-resolution VR Painting in Large Volumetric Canvas",
 * arXiv 1704.02724). All entry points are plain C: host or device pointers,
 * sizes and small structs; no C++ or PyTorch types cross this boundary.
 *
 * Threading and ownership: one global library context per process, bound to
 * the CUDA device that is current at the first canvox_upload_octree or
 * canvox_paint_spheres. Calls are not thread-safe; serialise them. The library
 * owns its device copy of the octree (and, for a painted canvas, the stamp
 * table), its camera staging buffers and its statistics buffer. The caller owns
 * every output buffer and every stream passed in.
 *
 * Errors: every int-returning call returns CANVOX_OK (0) or a negative
 * CANVOX_ERR_* code and sets a message readable with canvox_last_error().
 * No call aborts, throws or traps.
 */
#ifndef CANVOX_H
#define CANVOX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CANVOX_OK 0
#define CANVOX_ERR_INVALID_ARG (-1) /* bad pointer, size or option; nothing was launched */
#define CANVOX_ERR_NOT_UPLOADED (-2) /* render or hash before a successful upload */
#define CANVOX_ERR_BAD_TREE (-3)     /* upload validation failed; the previous canvas is kept */
#define CANVOX_ERR_CUDA (-4)         /* a CUDA runtime call failed (message has the CUDA error) */
#define CANVOX_ERR_OOM (-5)          /* device or pinned host allocation failed */
#define CANVOX_ERR_STEP_LIMIT (-6)   /* some ray hit the per-ray step limit (partial pixel written) */

#define CANVOX_PREC_MIXED 0 /* FP32 cell-local frames, FP64 rebase and error-budgeted FP64 boundaries */
#define CANVOX_PREC_FP64 1  /* plain FP64: canvas coordinates, leaf located from the root each step */
#define CANVOX_PREC_FP32 2  /* plain FP32 in canvas coordinates (the failing baseline of Sec. 6.3) */
#define CANVOX_PREC_CELL32 3  /* the paper's FP32 cell-local walk, p' s + c per step (Sec. 6.2-6.3) */
#define CANVOX_PREC_WORLD32 4 /* the same walk with the position in FP32 canvas coordinates (Sec. 6.3 comparison) */
#define CANVOX_PREC_CELL16 5  /* the cell-local walk with binary16 geometry (the half-precision remark of Sec. 6.3) */
#define CANVOX_PREC_FP64_LINKS 6 /* the mixed path's traversal (neighbour links, persistent queue) with every time,
                                    side test and sum in FP64: the precision comparator of the mixed path */

/*
 * One view (Sec. 6.1: the eye position is kept in FP64 canvas coordinates so
 * that stereo eyes do not snap to FP32 values). 136 bytes, no padding.
 *   eye, right, up, forward : canvas coordinates; right/up/forward need not be
 *       exactly orthonormal: the library orthonormalises them by Gram-Schmidt
 *       starting from forward, then up, then right.
 *   tan_half_fov_y : tangent of half the vertical field of view (> 0).
 *   width, height  : image size in pixels (>= 1 each, width * height < 2^31).
 *   out_offset_px  : index of this view's pixel (0,0) in the output image;
 *       pixel (i, j) (column i, row j from the top) is written at
 *       out_offset_px + j * width + i. Views must not overlap.
 *   background     : RGBA behind the canvas; the output is
 *       (C + T bg.rgb, 1 - T) with T the transmittance left at the end.
 * Pixel (i, j) shoots the ray through its centre:
 *   d = normalize(f + u r + v up), u = (2(i+1/2)/W - 1) tan * W/H,
 *   v = (1 - 2(j+1/2)/H) tan,
 * with f, up, r the orthonormalised frame. Every operation is IEEE FP64,
 * rounded separately (no fused multiply-add), in this order:
 *   x = (2i+1)/W - 1, y = 1 - (2j+1)/H, u = (x tan) (W/H), v = y tan,
 *   d = (f + u r) + v up, d /= sqrt((d0 d0 + d1 d1) + d2 d2).
 * A ray that lies exactly in a cell plane (a zero component of d, as in the
 * centre row or column of an axis-aligned view) then stays exactly in it, and
 * the side it runs on is the high side of that plane.
 */
typedef struct canvox_camera {
    double eye[3];
    double right[3];
    double up[3];
    double forward[3];
    double tan_half_fov_y;
    int32_t width;
    int32_t height;
    int64_t out_offset_px;
    float background[4];
} canvox_camera;

/*
 * Render options. Fill with canvox_default_opts() and change what you need.
 *   precision     : CANVOX_PREC_*.
 *   per_view      : 0 = all views in one persistent launch; 1 = one launch per view.
 *   use_graph     : 1 = replay the launch sequence from a cached CUDA graph.
 *   block_threads : threads per block of the persistent kernel (multiple of 32, 32..256).
 *   blocks_per_sm : persistent blocks per SM (the grid is SMs x this).
 *   refill        : a warp refetches rays when at most this many lanes are still busy (0..31).
 *   smem_records  : records of the breadth-first tree prefix (the top of the tree) copied to shared
 *                   memory at kernel start (0 = none, at most 6144; blocks per SM shrink to fit).
 *   frame_levels  : K, the most levels a local frame may sit above its cell (1..22).
 *   tile_w        : pixel tile a warp starts with: tile_w x (32 / tile_w), tile_w in {4, 8, 16, 32}.
 *   traversal     : 0 = neighbour links (the paper's neighbour graph, Sec. 4.1.1, built at upload),
 *                   1 = stack of ancestor records with re-descent from the common ancestor.
 *   step_limit    : most leaves one ray may visit (0 = 3 * 2^depth + 8, capped at 2^31 - 1).
 *   t_min         : stop a ray once its transmittance is below this (< 0: default 2^-20).
 *   err_budget    : per-ray bound on the colour error the FP32 boundaries may add before
 *                   the remaining boundaries are taken in FP64 (mixed precision only).
 *   step_count    : optional device int32 per output pixel: leaves visited by its ray.
 *   angle_deg     : optional device float per output pixel (CELL32 / WORLD32 / CELL16 only): angle in degrees
 *                   between the initial ray direction and the line from the eye to the ray's final
 *                   position (the ray-angle error of Sec. 6.3).
 *   count_reads   : 1 = count slot reads, leaf loads and record loads for canvox_stats (mixed precision);
 *                   0 = leave those three counters at 0 (a few instructions and registers less per leaf
 *                   step; the image is the same bit for bit).
 */
typedef struct canvox_render_opts {
    int32_t precision;
    int32_t per_view;
    int32_t use_graph;
    int32_t block_threads;
    int32_t blocks_per_sm;
    int32_t refill;
    int32_t smem_records;
    int32_t frame_levels;
    int32_t tile_w;
    int32_t traversal;
    int64_t step_limit;
    float t_min;
    float err_budget;
    int32_t* step_count;
    float* angle_deg;
    int32_t count_reads;
} canvox_render_opts;

/* Counters of the last completed render call (sums over all its rays). */
typedef struct canvox_stats {
    int64_t rays;            /* rays traced (pixels) */
    int64_t steps;           /* leaves visited */
    int64_t slot_reads;      /* child-slot reads a perfect stack needs: levels re-descended from the LCA */
    int64_t leaf_loads;      /* non-empty leaf values read (8 B each) */
    int64_t record_loads;    /* child-slot loads actually issued (stack restarts included) */
    int64_t fp64_boundaries; /* leaf boundaries whose crossing time was taken in FP64 */
    int64_t rebases;         /* local frames entered (FP64 rebase of the ray) */
    int64_t step_limited;    /* rays stopped by the step limit */
    int64_t h2d_bytes;       /* host-to-device bytes the call copied (view table) */
    int64_t d2h_bytes;       /* device-to-host bytes the call copied (image, canvox_render_host only) */
} canvox_stats;

/* Fill *o with the defaults (tuned values once canvox_autotune has run). */
void canvox_default_opts(canvox_render_opts* o);

/*
 * Validate and copy a canvas to the current CUDA device (synchronous).
 *   node_pool  : host int32[n_records][8], record 0 = root cell [-E/2, E/2]^3.
 *                Slot k of record r is child k = x + 2y + 4z (x, y, z = high
 *                half on that axis; Sec. 4.1.1: eight children per allocation
 *                unit, consecutive indices): v > 0 index of the child's record,
 *                v == 0 empty leaf (extinction 0), v < 0 a stored leaf. Stored
 *                leaves are numbered 0, 1, ... in breadth-first slot order
 *                (records in order, slots k = 0..7 within a record), and the
 *                slot holds -(number mod 2^31) - 1: below 2^31 leaves, -v-1 is
 *                the number itself; larger pools (up to 2^34 leaves) wrap.
 *   leaf_rgba  : host uint16[n_leaves][4], IEEE FP16 bits (R, G, B, sigma); sigma is
 *                the extinction per canvas unit (finite, >= 0); R, G, B finite.
 *                Leaf i is row i (n_leaves <= 2^34, n_records <= 2^31 - 1).
 *   depth      : deepest level allowed (1..30); the finest cell is extent * 2^-depth.
 *   extent     : canvas side (> 0, finite, at most 23 significant bits so that
 *                every cell plane is exact in FP64).
 * The upload also builds six neighbour links per record (48 bytes per record) for the
 * default traversal. Validation (CANVOX_ERR_BAD_TREE on failure, previous canvas kept): internal
 * children numbered 1, 2, ... in breadth-first order (each referenced once,
 * no cycles), leaves numbered 0, 1, ... in the same order (modulo 2^31), no record deeper
 * than depth - 1, leaf values finite with sigma >= 0. The host pools may be
 * freed on return. A 64-bit hash of the device copy is checked against the
 * host pools before the call returns.
 */
int canvox_upload_octree(const int32_t* node_pool, int64_t n_records, const uint16_t* leaf_rgba,
                         int64_t n_leaves, int32_t depth, double extent);

/*
 * Paint a canvas on the GPU and make it the current one (replaces canvox_upload_octree
 * for canvases built from spherical brush stamps; Sec. 5.1-5.2). Stamp i (applied in
 * order i = 0, 1, ...) is a sphere with centre centers[3i..3i+2] and radius radii[i]
 * (canvas units, host FP64) and brush value rgba[4i..4i+3] (host FP32 R, G, B, extinction).
 * Model: a stamp refines every cell it partially covers down to its target depth (the
 * smallest k with extent 2^-k <= r/10, at most depth; eight children copy the parent),
 * paints cells inside the sphere whole, paints partially covered cells at or below the
 * target depth by their centre, and descends into cells already refined. Paint blends
 * additively in FP32 (rgb' = B m + (1 - m) C, m = B_a / (B_a + C_a), a' = B_a + C_a).
 * Leaves are then clamped (rgb to [0, 1], extinction to [0, 60000]), rounded to FP16,
 * eight identical siblings merge bottom-up (the root stays), and the pools are written
 * in the breadth-first layout of canvox_upload_octree. The result is bit-identical to
 * painting the stamps one by one in that order. Synchronous; the previous canvas is
 * freed first (also on failure). Temporary device memory: per tree level, the ordered
 * stamp lists of the refined cells. n_records, n_leaves (optional) receive the pool
 * sizes. Errors: INVALID_ARG (non-finite input, negative radius or extinction, bad
 * depth/extent), OOM (device memory, or pools beyond 2^31 - 1 records or 2^34 leaves), CUDA.
 */
int canvox_paint_spheres(int32_t depth, double extent, const double* centers, const double* radii,
                         const float* rgba, int64_t n, int64_t* n_records, int64_t* n_leaves);

/*
 * Add n stamps after those already painted and repaint (the editing path: only the new
 * stamps, 56 bytes each, cross the bus; the painter keeps the stamp table of the current
 * canvas in device memory, and what it painted below level 5, per level-5 cell). Stamps
 * added later never change what earlier ones did, so only the level-5 cells whose stamp
 * lists the new stamps reach are painted again; the other cells' subtrees are kept. The
 * result is the canvas canvox_paint_spheres would build from the whole table. Needs a current canvas made by canvox_paint_spheres or this call
 * (CANVOX_ERR_NOT_UPLOADED otherwise, e.g. after canvox_upload_octree). Same arguments,
 * errors and synchronisation as canvox_paint_spheres; on an argument error nothing changes.
 */
int canvox_paint_append(const double* centers, const double* radii, const float* rgba, int64_t n,
                        int64_t* n_records, int64_t* n_leaves);

/* Sizes of the current canvas (any pointer may be NULL). */
int canvox_canvas_info(int64_t* n_records, int64_t* n_leaves, int32_t* depth, double* extent);

/*
 * Copy the current canvas to host memory in the layout of canvox_upload_octree:
 * node_pool int32[n_records][8], leaf_rgba uint16[n_leaves][4] (sizes from
 * canvox_canvas_info). Synchronous.
 */
int canvox_download_octree(int32_t* node_pool, uint16_t* leaf_rgba);

/*
 * Replace the values of leaves [first, first + count) of the current canvas with
 * leaf_rgba (host uint16[count][4], the layout of canvox_upload_octree); the tree
 * structure is unchanged. This is the dirty-range upload of a value edit (recolouring
 * or re-weighting paint without refining or merging cells, Sec. 4.1's editing of the
 * colour pool): only the changed range crosses the bus. The values are validated as at
 * upload (finite, extinction >= 0; CANVOX_ERR_BAD_TREE, nothing changed); the range
 * must lie in the pool (CANVOX_ERR_INVALID_ARG). Synchronous: waits for earlier
 * renders; the host-side pool hash is updated, so canvox_octree_hash still compares
 * the device copy with the values the caller supplied. A structural edit (cells
 * refined or merged) renumbers the breadth-first pools from the first change on:
 * upload again, or repaint with canvox_paint_append.
 */
int canvox_update_leaves(int64_t first, int64_t count, const uint16_t* leaf_rgba);

/*
 * Render n_views views into out_rgba_dev (device float32 RGBA, at least
 * max(out_offset_px + width * height) pixels, 16 bytes each), stream-ordered
 * on `stream` (a cudaStream_t; NULL = legacy default stream) with the default
 * options. Asynchronous: returns after enqueueing. `cams` is host memory and
 * may be freed on return. n_views == 0 is a no-op.
 */
int canvox_render(const canvox_camera* cams, int32_t n_views, float* out_rgba_dev, void* stream);

/* canvox_render with explicit options (opts == NULL: defaults). */
int canvox_render_ex(const canvox_camera* cams, int32_t n_views, float* out_rgba_dev, void* stream,
                     const canvox_render_opts* opts);

/*
 * Render into host memory: the image is produced in a library-owned device
 * buffer and copied to out_rgba_host (float32 RGBA, max(out_offset_px + W*H)
 * pixels; pinned memory copies fastest). Synchronous: returns when the host
 * buffer holds the image.
 */
int canvox_render_host(const canvox_camera* cams, int32_t n_views, float* out_rgba_host, void* stream,
                       const canvox_render_opts* opts);

/*
 * Render without allocating anything (the paper has no counterpart: this is
 * an interface for callers that cannot call cudaMalloc, such as code inside a
 * memory pool that owns all device memory, or a real-time loop that must not
 * touch the allocator). The caller passes its own device buffers:
 *   node_pool_dev, n_records, leaf_rgba_dev, n_leaves, depth, extent : the
 *       canvas in the layout of canvox_upload_octree, already in device memory
 *       and already valid under its rules (this call does not validate the
 *       pools; an invalid pool reads out of bounds);
 *   cams, n_views (0..64) : host camera records, as for canvox_render;
 *   out_rgba_dev, stream : as for canvox_render (asynchronous, stream-ordered).
 * Default options, no counters (canvox_get_stats does not see these calls).
 * The working memory (counters, ray-queue head, view table, eye paths) is one
 * fixed 24 KiB array in device global memory that every GPU loading the
 * library holds until the process exits. The first call on a device looks up
 * that array's device address and keeps it, so make it before any stream
 * capture, and do not reset the device (cudaDeviceReset) between calls in one
 * process: the kept address would then be stale. All
 * calls share the array: calls that overlap on the GPU race, so serialise
 * them (one stream, or wait between them). Each call first clears the
 * array's counters and queue head and stores its view table there with a
 * small kernel (the table travels as a kernel argument: no host buffer has to
 * outlive the call). More than 64 views, or n_records / n_leaves above
 * 2^31 - 1: CANVOX_ERR_INVALID_ARG. Step-limit overruns are not reported:
 * the limit is the default one (3 * 2^depth + 8 leaves per ray, capped at
 * 2^31 - 1), and every step crosses one plane of the finest grid that the ray
 * never crosses again, so a ray visits at most 3 * 2^depth - 2 leaves and
 * cannot reach the limit below depth 30.
 */
int canvox_render_noalloc(const int32_t* node_pool_dev, int64_t n_records, const uint16_t* leaf_rgba_dev,
                          int64_t n_leaves, int32_t depth, double extent, const canvox_camera* cams,
                          int32_t n_views, float* out_rgba_dev, void* stream);

/* Counters of the last render (synchronises with the library's work). */
int canvox_get_stats(canvox_stats* s);

/* 64-bit hashes of the uploaded pools: recomputed on the host copy and by a device kernel. */
int canvox_octree_hash(uint64_t* host_hash, uint64_t* device_hash);

/*
 * Search the schedule (block size, refill threshold, tile shape, shared-memory
 * prefix, frame levels, traversal; one parameter at a time, two passes) by timing renders
 * of these views, and keep the fastest as the default options. Synchronous. Writes the chosen options to *best when
 * best is not NULL.
 */
int canvox_autotune(const canvox_camera* cams, int32_t n_views, void* stream, canvox_render_opts* best);

/*
 * Measurement helpers (the paper reports no profile; these give the figures the
 * traversal is measured against). All are synchronous.
 *
 * canvox_footprint: the distinct records and stored leaves that the rays of these
 * views read, i.e. the compulsory bytes of a render from a cold cache
 * (32 * records + 8 * leaves). Marked by the plain FP64 traversal (leaf located
 * from the root each step, so every ancestor of every visited leaf counts once),
 * with the default t_min and no step limit. Needs an uploaded canvas; overwrites
 * the counters that canvox_get_stats reports. Temporary device memory: one bit per
 * record and per leaf.
 */
int canvox_footprint(const canvox_camera* cams, int32_t n_views, void* stream, int64_t* n_records,
                     int64_t* n_leaves);

/*
 * canvox_probe_l2_gather: bandwidth of random 32-byte sector gathers served by L2
 * (loads that bypass L1, from a buffer of buffer_bytes rounded down to a power of
 * two; 0 = half the device's L2), in GB/s counted at 32 bytes per gather. The
 * access pattern of the record and leaf loads with DRAM taken out. buffer_bytes
 * in [32 KiB, 64 GiB] (or 0), else CANVOX_ERR_INVALID_ARG.
 */
int canvox_probe_l2_gather(int64_t buffer_bytes, double* sector_gbs);

/* canvox_probe_fp64: FP64 FMA throughput of the device (independent chains), GFLOP/s (2 per FMA). */
int canvox_probe_fp64(double* gflops);

/* Message of the last error on the calling thread ("" if none). */
const char* canvox_last_error(void);

/* Free every device and pinned allocation of the library (safe to call twice). */
void canvox_release(void);

#ifdef __cplusplus
}
#endif

#endif /* CANVOX_H */
