// Internal types shared by the CUDA translation units of libcanvox.so.
#pragma once

#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/canvox.h"

namespace canvox {

// Rays are handed out in tiles of tw x th = 32 pixels (one warp; tw = 2^tile_wl);
// a view of W x H pixels has ceil(W/tw) x ceil(H/th) tiles, and ray g of the
// launch is lane g % 32 of tile g / 32.
constexpr int kMaxDepth = 30;
constexpr int kMaxSmemRecords = 6144;
// Leaves are numbered in breadth-first slot order; a slot holds the number modulo 2^31 (-v - 1 for
// v < 0). The number passes a multiple of 2^31 at most kMaxWraps times: pools of up to 8 x 2^31 leaves.
constexpr int kMaxWraps = 7;
constexpr int64_t kMaxLeaves = (int64_t)(kMaxWraps + 1) << 31;

// Device view of the uploaded canvas.
struct Tree {
    const int32_t* nodes;  // n_rec x 8 child slots
    const uint2* ropes;    // n_rec x 6 face neighbours (null: none built), see rope_level_kernel
    const uint2* leaves;   // n_leaf x FP16 (R,G | B,sigma)
    int64_t n_rec;
    int64_t n_leaf;
    int32_t depth;
    int32_t n_wrap;  // multiples of 2^31 the leaf numbers pass
    double extent;
    double half;  // extent / 2
    int64_t wrap[kMaxWraps];  // slot position 8 r + k of leaf m 2^31 (m = 1 .. n_wrap), increasing
};

// Number of the leaf in slot k of record rec, whose value is v < 0: the slot holds its low 31 bits
// (-v - 1); each wrap position at or before this slot adds 2^31.
__host__ __device__ __forceinline__ int64_t leaf_index(const Tree& t, int64_t rec, int k, int32_t v) {
    int64_t li = -((int64_t)v + 1);
    if (t.n_wrap > 0) {
        const int64_t pos = rec * 8 + k;
        for (int m = 0; m < t.n_wrap; ++m) li += pos >= t.wrap[m] ? ((int64_t)1 << 31) : 0;
    }
    return li;
}

// Per-view set-up, computed on the host in FP64 from canvox_camera (host code is
// compiled without contraction, so the frame is the one the camera model defines).
struct View {
    double eye[3];
    double f[3], u[3], r[3];  // orthonormal frame (Gram-Schmidt from forward)
    double sx, sy;            // tan * aspect, tan
    double aspect;            // width / height
    double two_over_w, two_over_h;
    float bg[4];
    int64_t out_offset;
    int64_t ray_begin;  // first ray index of this view in the launch (multiple of 32)
    int32_t width, height;
    int32_t tiles_x;
    int32_t tile_wl;  // log2 of the tile width
};

// Leaf holding the eye of a view, located once per render by eye_path_kernel.
// Valid (len > 0) when the eye is inside the canvas and on no cell plane of its
// path: every ray of the view then starts in this leaf at t = 0 (the ray is on
// the high side of a plane just after t = 0 iff the eye is above it).
struct EyePath {
    int32_t rec[kMaxDepth + 1];  // record of each ancestor level 0 .. len-1
    uint32_t c[3];               // leaf coordinates at level len
    int32_t len;                 // leaf level (0: not valid, trace from the root)
    uint2 val;                   // leaf value (0, 0 = empty)
    int32_t stored;              // 1 if the leaf has a stored value (slot < 0)
    int32_t pad[2];
};

// Counters, in the order of canvox_stats.
enum Stat {
    kStatRays = 0,
    kStatSteps,
    kStatSlotReads,
    kStatLeafLoads,
    kStatRecordLoads,
    kStatFp64Boundaries,
    kStatRebases,
    kStatStepLimited,
    kNumStats
};

// Device scratch: ray queue heads, counters, status word (zeroed before a launch).
struct Scratch {
    unsigned long long stats[kNumStats];
    unsigned long long status;
    unsigned long long queue[1];  // one head per launch (per view in per-view mode)
};

struct MixedParams {
    Tree tree;
    const View* views;
    const EyePath* eye;  // one per view
    int32_t n_views;
    int32_t refill;
    int64_t total_rays;  // the queue hands out rays [0, total_rays) ...
    int64_t ray_base;    // ... which are rays ray_base + g of the view table
    float4* out;
    int32_t* step_count;
    unsigned long long* queue;
    Scratch* scratch;
    int64_t step_limit;
    float t_min;
    float err_budget;
    int32_t frame_levels;
    int32_t smem_records;
    int32_t use_ropes;   // 1: neighbour links (Tree::ropes), 0: stack of ancestors
    int32_t count_reads; // 1: count slot reads, leaf loads and record loads (canvox_stats)
};

struct PlainParams {
    Tree tree;
    const View* view;  // one view per launch
    float4* out;
    int32_t* step_count;
    float* angle_deg;  // per-pixel ray-angle error (single-precision traversals of the paper only)
    Scratch* scratch;
    int64_t step_limit;
    float t_min;
    uint32_t* mark_rec;   // footprint bitsets (plain kernel only; null: off): the record holding
    uint32_t* mark_leaf;  // each located leaf's slot, and each stored leaf loaded
};

// Launchers (trace_mixed.cu, trace_plain.cu, runtime.cu).
cudaError_t launch_mixed(const MixedParams& p, int grid, int block, cudaStream_t s);  // smem from p.smem_records
cudaError_t mixed_max_blocks_per_sm(int block, int smem_bytes, int* out);
cudaError_t launch_fp64links(const MixedParams& p, int grid, int block, cudaStream_t s);  // needs p.tree.ropes
cudaError_t fp64links_max_blocks_per_sm(int block, int* out);
cudaError_t launch_plain(const PlainParams& p, int precision, long long n_pixels, cudaStream_t s);
cudaError_t launch_local32(const PlainParams& p, int precision, long long n_pixels, cudaStream_t s);
cudaError_t launch_hash(const Tree& t, unsigned long long* out, cudaStream_t s);
cudaError_t launch_rope_level(const int32_t* nodes, uint2* ropes, int64_t lo, int64_t hi, int level, cudaStream_t s);
cudaError_t launch_eye_paths(const Tree& t, const View* views, int n_views, EyePath* out, cudaStream_t s);
cudaError_t probe_l2_gather(int64_t buffer_bytes, double* gbs);
cudaError_t probe_fp64(double* gflops);
// The device painter. *cache: what it keeps of the last painted canvas for appends (null: none). When it holds
// the same depth and extent and the first stamps of this table, only the partitions whose stamp lists changed
// are painted again; either way it is replaced by the new canvas's cache (null on failure).
struct PaintCache;
void paint_cache_free(PaintCache* c);
cudaError_t paint_pools(int32_t depth, double extent, const double* d_centers, const double* d_radii, const float4* d_rgba,
                        int64_t n, PaintCache** cache, int32_t** d_nodes, uint2** d_leaves, int64_t* n_rec,
                        int64_t* n_leaf, std::vector<int64_t>* level_begin, int64_t* wrap, int32_t* n_wrap);  // wrap: kMaxWraps
cudaError_t scan_i64(int64_t* d, int64_t n, int64_t* total);
cudaError_t footprint_finish(const int32_t* nodes, const int64_t* level_begin, int n_levels, uint32_t* rec_bits,
                             int64_t rec_words, const uint32_t* leaf_bits, int64_t leaf_words,
                             unsigned long long* d_count, int64_t* n_records, int64_t* n_leaves);

// Host helpers of runtime.cu shared with other entry points.
int build_views(const canvox_camera* cams, int n, int tile_w, View* out, int64_t* total_rays);
void builtin_render_opts(canvox_render_opts* o);
int set_error(int code, const char* msg);
void clear_error();

// 64-bit element hash shared by the host and device hash of the pools.
__host__ __device__ inline unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__host__ __device__ inline unsigned long long elem_hash(unsigned long long tag, unsigned long long index,
                                                        unsigned long long value) {
    return mix64(tag ^ mix64(index * 0x9E3779B97F4A7C15ull + value));
}

}  // namespace canvox

namespace canvox {
// Unit direction of the ray through the centre of pixel (i, j) of view V, in
// IEEE FP64 with every operation rounded separately in the order the camera
// model of include/canvox.h fixes:
//   x = (2i+1)/W - 1,  y = 1 - (2j+1)/H,  u = (x tan) aspect,  v = y tan,
//   d = (f + u r) + v up,  d /= sqrt((d0 d0 + d1 d1) + d2 d2).
// A ray that lies exactly in a cell plane (d_a == 0) must come out exactly so,
// since the side of the plane it runs on is decided by this value.
__device__ __forceinline__ void pixel_ray(const View& V, int i, int j, double d[3]) {
    const double x = __dadd_rn(__ddiv_rn(2.0 * i + 1.0, (double)V.width), -1.0);
    const double y = __dsub_rn(1.0, __ddiv_rn(2.0 * j + 1.0, (double)V.height));
    const double u = __dmul_rn(__dmul_rn(x, V.sy), V.aspect);
    const double v = __dmul_rn(y, V.sy);
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = __dadd_rn(__dadd_rn(V.f[a], __dmul_rn(u, V.r[a])), __dmul_rn(v, V.u[a]));
    const double n = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2])));
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = __ddiv_rn(d[a], n);
}
}  // namespace canvox
