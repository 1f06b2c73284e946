// libcanvox.so runtime: the C ABI of include/canvox.h.
//
// Host side of the renderer: canvas validation and upload (Sec. 4.1: linear
// index pools, eight children per allocation unit, copied to the GPU), the
// host/device bit-identity hash, per-view FP64 set-up of the eye and pixel
// grid (Sec. 6.1), launch of the traversal kernels, CUDA-graph replay,
// counters, the schedule autotuner, the device painter's stamp table and the
// measurement helpers' set-up.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "canvox_internal.cuh"

using namespace canvox;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    cudaGetLastError();  // clear a sticky launch error if it is not a context error
    return fail(e == cudaErrorMemoryAllocation ? CANVOX_ERR_OOM : CANVOX_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define CK(call, what)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

struct GraphEntry {
    bool valid = false;
    int buf = 0;
    const void* out = nullptr;
    int32_t n_views = 0;
    int64_t total_rays = 0;
    unsigned long long layout = 0;  // hash of every view's size and offset
    canvox_render_opts opts{};
    cudaGraphExec_t exec = nullptr;
};

struct Ctx {
    int device = -1;
    int sm_count = 0;
    // canvas
    int32_t* d_nodes = nullptr;
    uint2* d_leaves = nullptr;
    uint2* d_ropes = nullptr;
    int64_t n_rec = 0, n_leaf = 0;
    int32_t depth = 0;
    double extent = 0.0;
    int32_t n_wrap = 0;             // leaf numbers pass a multiple of 2^31 this many times ...
    int64_t wrap[kMaxWraps] = {};   // ... at these slot positions 8 r + k
    unsigned long long host_hash = 0;
    std::vector<int64_t> level_begin;  // records of level l: [level_begin[l], level_begin[l + 1])
    bool uploaded = false;
    // stamp table of a painted canvas (kept on the device for canvox_paint_append)
    double* d_st_c = nullptr;
    double* d_st_r = nullptr;
    float4* d_st_rgba = nullptr;
    int64_t st_n = 0, st_cap = 0;
    bool painted = false;
    PaintCache* paint_cache = nullptr;  // the painter's state of the current painted canvas (for appends)
    // views: device table and two pinned staging buffers, each guarded by an event
    View* d_views = nullptr;
    EyePath* d_eye = nullptr;
    int views_cap = 0;
    View* h_views[2] = {nullptr, nullptr};
    cudaEvent_t staged[2] = {nullptr, nullptr};
    int next_buf = 0;
    // scratch: counters, status and one queue head per launch
    Scratch* d_scratch = nullptr;
    int scratch_queues = 0;
    unsigned long long* d_hash = nullptr;
    cudaEvent_t done = nullptr;  // recorded after every render
    bool any_render = false;
    int64_t last_h2d = 0, last_d2h = 0;
    // host render target
    float4* d_host_out = nullptr;
    int64_t host_out_cap = 0;
    // defaults (autotuned)
    canvox_render_opts tuned{};
    bool have_tuned = false;
    GraphEntry graphs[4];
    int graph_next = 0;
};

Ctx g;

size_t scratch_bytes(int queues) { return sizeof(Scratch) + sizeof(unsigned long long) * (size_t)(queues > 1 ? queues - 1 : 0); }

void builtin_defaults(canvox_render_opts* o) {
    std::memset(o, 0, sizeof(*o));
    o->precision = CANVOX_PREC_MIXED;
    o->per_view = 0;
    o->use_graph = 0;
    o->block_threads = 256;
    o->blocks_per_sm = 0;
    o->refill = 0;
    o->smem_records = 0;
    o->frame_levels = 20;
    o->tile_w = 8;
    o->traversal = 0;
    o->step_limit = 0;
    o->t_min = -1.0f;
    o->err_budget = 3.0e-6f;
    o->step_count = nullptr;
    o->angle_deg = nullptr;
    o->count_reads = 1;
}

int ensure_device() {
    int dev;
    CK(cudaGetDevice(&dev), "cudaGetDevice");
    if (g.device >= 0 && g.device != dev)
        return fail(CANVOX_ERR_INVALID_ARG, "canvas was uploaded on device %d, current device is %d", g.device, dev);
    if (g.device < 0) {
        g.device = dev;
        CK(cudaDeviceGetAttribute(&g.sm_count, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute");
        CK(cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming), "cudaEventCreate");
        for (int b = 0; b < 2; ++b) CK(cudaEventCreateWithFlags(&g.staged[b], cudaEventDisableTiming), "cudaEventCreate");
        CK(cudaMalloc(&g.d_hash, sizeof(unsigned long long)), "cudaMalloc(hash)");
    }
    return CANVOX_OK;
}

void drop_graphs() {
    for (auto& e : g.graphs) {
        if (e.exec) cudaGraphExecDestroy(e.exec);
        e = GraphEntry();
    }
}

int ensure_views(int n) {
    if (n <= g.views_cap) return CANVOX_OK;
    int cap = 64;
    while (cap < n) cap *= 2;
    // wait for every user of the old buffers, then grow
    if (g.any_render) CK(cudaEventSynchronize(g.done), "cudaEventSynchronize");
    drop_graphs();
    if (g.d_views) cudaFree(g.d_views);
    if (g.d_eye) cudaFree(g.d_eye);
    for (int b = 0; b < 2; ++b)
        if (g.h_views[b]) cudaFreeHost(g.h_views[b]);
    g.d_views = nullptr;
    g.d_eye = nullptr;
    g.h_views[0] = g.h_views[1] = nullptr;
    g.views_cap = 0;
    CK(cudaMalloc(&g.d_views, sizeof(View) * (size_t)cap), "cudaMalloc(views)");
    CK(cudaMalloc(&g.d_eye, sizeof(EyePath) * (size_t)cap), "cudaMalloc(eye paths)");
    for (int b = 0; b < 2; ++b) CK(cudaMallocHost(&g.h_views[b], sizeof(View) * (size_t)cap), "cudaMallocHost(views)");
    g.views_cap = cap;
    return CANVOX_OK;
}

int ensure_scratch(int queues) {
    if (queues <= g.scratch_queues) return CANVOX_OK;
    int cap = 64;
    while (cap < queues) cap *= 2;
    if (g.any_render) CK(cudaEventSynchronize(g.done), "cudaEventSynchronize");
    drop_graphs();
    if (g.d_scratch) cudaFree(g.d_scratch);
    g.d_scratch = nullptr;
    g.scratch_queues = 0;
    CK(cudaMalloc(&g.d_scratch, scratch_bytes(cap)), "cudaMalloc(scratch)");
    CK(cudaMemset(g.d_scratch, 0, scratch_bytes(cap)), "cudaMemset(scratch)");
    g.scratch_queues = cap;
    return CANVOX_OK;
}

bool finite3(const double* v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }
double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// Per-view set-up in FP64: Gram-Schmidt frame from forward, pixel scale factors, tiling.
int setup_views(const canvox_camera* cams, int n, int tile_w, View* out, int64_t* total_rays) {
    const int wl = tile_w == 4 ? 2 : tile_w == 8 ? 3 : tile_w == 16 ? 4 : 5;
    const int tw = 1 << wl, th = 32 >> wl;
    int64_t ray = 0;
    for (int v = 0; v < n; ++v) {
        const canvox_camera& c = cams[v];
        if (c.width < 1 || c.height < 1 || !(c.tan_half_fov_y > 0.0) || !std::isfinite(c.tan_half_fov_y) ||
            c.out_offset_px < 0 || !finite3(c.eye) || !finite3(c.right) || !finite3(c.up) || !finite3(c.forward))
            return fail(CANVOX_ERR_INVALID_ARG, "camera %d: bad size, field of view, offset or non-finite vector", v);
        for (int a = 0; a < 4; ++a)
            if (!std::isfinite(c.background[a])) return fail(CANVOX_ERR_INVALID_ARG, "camera %d: non-finite background", v);
        if ((int64_t)c.width * c.height > 0x7FFFFFFFll)
            return fail(CANVOX_ERR_INVALID_ARG, "camera %d: more than 2^31 - 1 pixels", v);
        View& V = out[v];
        std::memset(&V, 0, sizeof(V));
        double n0 = std::sqrt(dot3(c.forward, c.forward));
        if (!(n0 > 0.0)) return fail(CANVOX_ERR_INVALID_ARG, "camera %d: zero forward vector", v);
        for (int a = 0; a < 3; ++a) V.f[a] = c.forward[a] / n0;
        const double uf = dot3(c.up, V.f);
        for (int a = 0; a < 3; ++a) V.u[a] = c.up[a] - uf * V.f[a];
        double n1 = std::sqrt(dot3(V.u, V.u));
        if (!(n1 > 0.0)) return fail(CANVOX_ERR_INVALID_ARG, "camera %d: up is parallel to forward", v);
        for (int a = 0; a < 3; ++a) V.u[a] /= n1;
        const double rf = dot3(c.right, V.f), ru = dot3(c.right, V.u);
        for (int a = 0; a < 3; ++a) V.r[a] = c.right[a] - rf * V.f[a] - ru * V.u[a];
        double n2 = std::sqrt(dot3(V.r, V.r));
        if (!(n2 > 0.0)) return fail(CANVOX_ERR_INVALID_ARG, "camera %d: right is in the forward/up plane", v);
        for (int a = 0; a < 3; ++a) V.r[a] /= n2;
        for (int a = 0; a < 3; ++a) V.eye[a] = c.eye[a];
        V.sy = c.tan_half_fov_y;
        V.aspect = (double)c.width / (double)c.height;
        V.sx = c.tan_half_fov_y * V.aspect;
        V.two_over_w = 2.0 / (double)c.width;
        V.two_over_h = 2.0 / (double)c.height;
        for (int a = 0; a < 4; ++a) V.bg[a] = c.background[a];
        V.out_offset = c.out_offset_px;
        V.width = c.width;
        V.height = c.height;
        V.tiles_x = (c.width + tw - 1) / tw;
        V.tile_wl = wl;
        const int64_t tiles = (int64_t)V.tiles_x * ((c.height + th - 1) / th);
        V.ray_begin = ray;
        ray += tiles * 32;
    }
    *total_rays = ray;
    return CANVOX_OK;
}

int resolve_opts(const canvox_render_opts* in, canvox_render_opts* o) {
    if (in) *o = *in;
    else canvox_default_opts(o);
    if (o->precision < 0 || o->precision > 6) return fail(CANVOX_ERR_INVALID_ARG, "precision %d", o->precision);
    if (o->block_threads == 0) o->block_threads = 256;
    if (o->block_threads < 32 || o->block_threads > 256 || o->block_threads % 32)
        return fail(CANVOX_ERR_INVALID_ARG, "block_threads %d (multiple of 32, at most 256)", o->block_threads);
    if (o->refill < 0 || o->refill > 31) return fail(CANVOX_ERR_INVALID_ARG, "refill %d (0..31)", o->refill);
    if (o->frame_levels == 0) o->frame_levels = 20;
    if (o->frame_levels < 1 || o->frame_levels > 22) return fail(CANVOX_ERR_INVALID_ARG, "frame_levels %d (1..22)", o->frame_levels);
    if (o->blocks_per_sm < 0 || o->smem_records < 0 || o->step_limit < 0)
        return fail(CANVOX_ERR_INVALID_ARG, "negative schedule option");
    if (o->smem_records > kMaxSmemRecords) return fail(CANVOX_ERR_INVALID_ARG, "smem_records %d (at most 6144)", o->smem_records);
    if (o->smem_records > g.n_rec) o->smem_records = (int32_t)g.n_rec;
    if (o->tile_w == 0) o->tile_w = 8;
    if (o->tile_w != 4 && o->tile_w != 8 && o->tile_w != 16 && o->tile_w != 32)
        return fail(CANVOX_ERR_INVALID_ARG, "tile_w %d (4, 8, 16 or 32)", o->tile_w);
    if (o->traversal != 0 && o->traversal != 1) return fail(CANVOX_ERR_INVALID_ARG, "traversal %d (0 or 1)", o->traversal);
    if (o->count_reads != 0 && o->count_reads != 1) return fail(CANVOX_ERR_INVALID_ARG, "count_reads %d (0 or 1)", o->count_reads);
    if (!(o->err_budget >= 0.0f) || !std::isfinite(o->err_budget)) return fail(CANVOX_ERR_INVALID_ARG, "err_budget");
    if (!std::isfinite(o->t_min)) return fail(CANVOX_ERR_INVALID_ARG, "t_min");
    if (o->t_min < 0.0f) o->t_min = 9.5367431640625e-07f;  // 2^-20
    if (o->step_limit == 0) {
        const int64_t lim = 3 * ((int64_t)1 << g.depth) + 8;
        o->step_limit = lim > 0x7FFFFFFF ? 0x7FFFFFFF : lim;
    }
    if (o->blocks_per_sm == 0) {
        int b = 0;
        CK(mixed_max_blocks_per_sm(o->block_threads, o->smem_records * 32, &b), "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
        o->blocks_per_sm = b > 0 ? b : 1;
    }
    return CANVOX_OK;
}

Tree device_tree() {
    Tree t;
    t.nodes = g.d_nodes;
    t.ropes = g.d_ropes;
    t.leaves = g.d_leaves;
    t.n_rec = g.n_rec;
    t.n_leaf = g.n_leaf;
    t.depth = g.depth;
    t.n_wrap = g.n_wrap;
    for (int m = 0; m < kMaxWraps; ++m) t.wrap[m] = g.wrap[m];
    t.extent = g.extent;
    t.half = 0.5 * g.extent;
    return t;
}

// The launch sequence of one render: stage views, clear scratch, trace.
int enqueue(const View* hv, const View* views_host, int n, int64_t total_rays, float* out,
            const canvox_render_opts& o, cudaStream_t s) {
    const int queues = o.per_view ? n : 1;
    CK(cudaMemcpyAsync(g.d_views, hv, sizeof(View) * (size_t)n, cudaMemcpyHostToDevice, s), "cudaMemcpyAsync(views)");
    CK(cudaMemsetAsync(g.d_scratch, 0, scratch_bytes(queues), s), "cudaMemsetAsync(scratch)");
    const Tree t = device_tree();
    if (o.precision == CANVOX_PREC_MIXED || o.precision == CANVOX_PREC_FP64_LINKS) {
        // the persistent traversal: mixed precision, or its FP64 twin (same traversal, FP64 arithmetic)
        const bool f64 = o.precision == CANVOX_PREC_FP64_LINKS;
        int bps = o.blocks_per_sm;
        if (f64) {
            int b = 0;
            CK(fp64links_max_blocks_per_sm(o.block_threads, &b), "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
            bps = b > 0 ? (b < bps ? b : bps) : 1;
        }
        auto launch = [&](const MixedParams& p, int grid) {
            return f64 ? launch_fp64links(p, grid, o.block_threads, s) : launch_mixed(p, grid, o.block_threads, s);
        };
        CK(launch_eye_paths(t, g.d_views, n, g.d_eye, s), "eye path kernel launch");
        MixedParams p;
        std::memset(&p, 0, sizeof(p));
        p.tree = t;
        p.out = reinterpret_cast<float4*>(out);
        p.step_count = o.step_count;
        p.scratch = g.d_scratch;
        p.step_limit = o.step_limit;
        p.t_min = o.t_min;
        p.err_budget = o.err_budget;
        p.frame_levels = o.frame_levels;
        p.refill = o.refill;
        p.smem_records = o.smem_records;
        p.use_ropes = o.traversal == 0 ? 1 : 0;
        p.count_reads = o.count_reads;
        if (!o.per_view) {
            p.views = g.d_views;
            p.eye = g.d_eye;
            p.n_views = n;
            p.total_rays = total_rays;
            p.ray_base = 0;
            p.queue = g.d_scratch->queue;
            const int grid = g.sm_count * bps;
            CK(launch(p, grid), "traversal kernel launch");
        } else {
            for (int v = 0; v < n; ++v) {
                p.views = g.d_views + v;
                p.eye = g.d_eye + v;
                p.n_views = 1;
                const int64_t rays = (v + 1 < n ? views_host[v + 1].ray_begin : total_rays) - views_host[v].ray_begin;
                p.total_rays = rays;
                p.ray_base = views_host[v].ray_begin;
                p.queue = g.d_scratch->queue + v;
                int64_t blocks = (rays + o.block_threads - 1) / o.block_threads;
                int64_t cap = (int64_t)g.sm_count * bps;
                const int grid = (int)(blocks < cap ? blocks : cap);
                CK(launch(p, grid > 0 ? grid : 1), "traversal kernel launch");
            }
        }
    } else {
        PlainParams p;
        std::memset(&p, 0, sizeof(p));
        p.tree = t;
        p.out = reinterpret_cast<float4*>(out);
        p.step_count = o.step_count;
        p.scratch = g.d_scratch;
        p.step_limit = o.step_limit;
        p.t_min = o.t_min;
        p.angle_deg = o.angle_deg;
        for (int v = 0; v < n; ++v) {
            p.view = g.d_views + v;
            const long long npx = (long long)views_host[v].width * views_host[v].height;
            if (o.precision == CANVOX_PREC_CELL32 || o.precision == CANVOX_PREC_WORLD32 || o.precision == CANVOX_PREC_CELL16)
                CK(launch_local32(p, o.precision, npx, s), "single-precision walk launch");
            else
                CK(launch_plain(p, o.precision, npx, s), "plain kernel launch");
        }
    }
    return CANVOX_OK;
}

bool same_opts(const canvox_render_opts& a, const canvox_render_opts& b) { return std::memcmp(&a, &b, sizeof(a)) == 0; }

int check_canvas_args(int32_t depth, double extent) {
    if (depth < 1 || depth > kMaxDepth) return fail(CANVOX_ERR_INVALID_ARG, "depth %d not in 1..30", depth);
    if (!(extent > 0.0) || !std::isfinite(extent)) return fail(CANVOX_ERR_INVALID_ARG, "extent must be finite and > 0");
    int ex;
    const double m = std::frexp(extent, &ex);  // m in [0.5, 1)
    const double scaled = std::ldexp(m, 23);  // integer iff at most 23 significant bits
    if (scaled != std::floor(scaled))
        return fail(CANVOX_ERR_INVALID_ARG, "extent %.17g has more than 23 significant bits", extent);
    return CANVOX_OK;
}

// Wait for every render, then free the current canvas (pools and links).
int drop_canvas() {
    if (g.any_render) CK(cudaEventSynchronize(g.done), "cudaEventSynchronize");
    drop_graphs();
    if (g.d_nodes) cudaFree(g.d_nodes);
    if (g.d_leaves) cudaFree(g.d_leaves);
    if (g.d_ropes) cudaFree(g.d_ropes);
    g.d_nodes = nullptr;
    g.d_leaves = nullptr;
    g.d_ropes = nullptr;
    g.uploaded = false;
    g.painted = false;
    return CANVOX_OK;
}

// Room for n stamps in the device stamp table (keeps the first `keep` rows).
int reserve_stamps(int64_t n, int64_t keep) {
    if (n <= g.st_cap) return CANVOX_OK;
    int64_t cap = 1024;
    while (cap < n) cap *= 2;
    double *c = nullptr, *r = nullptr;
    float4* q = nullptr;
    cudaError_t e = cudaMalloc(&c, sizeof(double) * 3 * (size_t)cap);
    if (e == cudaSuccess) e = cudaMalloc(&r, sizeof(double) * (size_t)cap);
    if (e == cudaSuccess) e = cudaMalloc(&q, sizeof(float4) * (size_t)cap);
    if (e == cudaSuccess && keep > 0) e = cudaMemcpy(c, g.d_st_c, sizeof(double) * 3 * (size_t)keep, cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess && keep > 0) e = cudaMemcpy(r, g.d_st_r, sizeof(double) * (size_t)keep, cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess && keep > 0) e = cudaMemcpy(q, g.d_st_rgba, sizeof(float4) * (size_t)keep, cudaMemcpyDeviceToDevice);
    if (e != cudaSuccess) {
        cudaFree(c);
        cudaFree(r);
        cudaFree(q);
        return cuda_fail(e, "stamp table");
    }
    cudaFree(g.d_st_c);
    cudaFree(g.d_st_r);
    cudaFree(g.d_st_rgba);
    g.d_st_c = c;
    g.d_st_r = r;
    g.d_st_rgba = q;
    g.st_cap = cap;
    return CANVOX_OK;
}

int check_stamps(const double* centers, const double* radii, const float* rgba, int64_t n) {
    if (n < 0 || (n > 0 && (!centers || !radii || !rgba)) || n >= 0x7FFFFFFFll)
        return fail(CANVOX_ERR_INVALID_ARG, "null stamp arrays or bad count");
    for (int64_t i = 0; i < n; ++i) {
        if (!std::isfinite(centers[3 * i]) || !std::isfinite(centers[3 * i + 1]) || !std::isfinite(centers[3 * i + 2]) ||
            !std::isfinite(radii[i]) || radii[i] < 0.0)
            return fail(CANVOX_ERR_INVALID_ARG, "stamp %lld: non-finite centre or bad radius", (long long)i);
        for (int c = 0; c < 4; ++c)
            if (!std::isfinite(rgba[4 * i + c])) return fail(CANVOX_ERR_INVALID_ARG, "stamp %lld: non-finite colour", (long long)i);
        if (rgba[4 * i + 3] < 0.0f) return fail(CANVOX_ERR_INVALID_ARG, "stamp %lld: negative extinction", (long long)i);
    }
    return CANVOX_OK;
}


// Neighbour links of the current pools, one launch per level (parents first).
int build_links() {
    CK(cudaMalloc(&g.d_ropes, sizeof(uint2) * 6 * (size_t)g.n_rec), "cudaMalloc(ropes)");
    for (size_t l = 0; l + 1 < g.level_begin.size(); ++l)
        CK(launch_rope_level(g.d_nodes, g.d_ropes, g.level_begin[l], g.level_begin[l + 1], (int)l, 0), "rope kernel launch");
    CK(cudaDeviceSynchronize(), "rope build");
    return CANVOX_OK;
}

// Paint the device stamp table into new pools and make them the current canvas.
int paint_table(int32_t depth, double extent, int64_t* n_records, int64_t* n_leaves) {
    int32_t* nodes = nullptr;
    uint2* leaves = nullptr;
    int64_t nr = 0, nl = 0;
    std::vector<int64_t> lb;
    int64_t wraps[kMaxWraps] = {};
    int32_t n_wrap = 0;
    CK(paint_pools(depth, extent, g.d_st_c, g.d_st_r, g.d_st_rgba, g.st_n, &g.paint_cache, &nodes, &leaves, &nr, &nl, &lb,
                   wraps, &n_wrap),
       "device painter (or a canvas beyond 2^31 - 1 records / 2^34 leaves)");
    g.d_nodes = nodes;
    g.d_leaves = leaves;
    g.n_wrap = n_wrap;
    for (int m = 0; m < kMaxWraps; ++m) g.wrap[m] = m < n_wrap ? wraps[m] : 0;
    g.n_rec = nr;
    g.n_leaf = nl;
    g.depth = depth;
    g.extent = extent;
    g.level_begin = lb;
    // no host copy exists: the device hash stands for both
    CK(cudaMemset(g.d_hash, 0, sizeof(unsigned long long)), "cudaMemset(hash)");
    CK(launch_hash(device_tree(), g.d_hash, 0), "hash kernel launch");
    CK(cudaMemcpy(&g.host_hash, g.d_hash, sizeof(unsigned long long), cudaMemcpyDeviceToHost), "cudaMemcpy(hash)");
    int rc = build_links();
    if (rc) return rc;
    g.uploaded = true;
    g.painted = true;
    if (n_records) *n_records = nr;
    if (n_leaves) *n_leaves = nl;
    return CANVOX_OK;
}

}  // namespace

namespace canvox {
int build_views(const canvox_camera* cams, int n, int tile_w, View* out, int64_t* total_rays) {
    return setup_views(cams, n, tile_w, out, total_rays);
}
void builtin_render_opts(canvox_render_opts* o) { builtin_defaults(o); }
int set_error(int code, const char* msg) { return fail(code, "%s", msg); }
void clear_error() { g_err.clear(); }
}  // namespace canvox

extern "C" {

void canvox_default_opts(canvox_render_opts* o) {
    if (!o) return;
    if (g.have_tuned) *o = g.tuned;
    else builtin_defaults(o);
}

const char* canvox_last_error(void) { return g_err.c_str(); }

int canvox_upload_octree(const int32_t* node_pool, int64_t n_records, const uint16_t* leaf_rgba, int64_t n_leaves,
                         int32_t depth, double extent) {
    g_err.clear();
    if (!node_pool || n_records < 1 || n_leaves < 0 || (n_leaves > 0 && !leaf_rgba))
        return fail(CANVOX_ERR_INVALID_ARG, "null pool or bad count");
    if (n_records > 0x7FFFFFFFll || n_leaves > kMaxLeaves)
        return fail(CANVOX_ERR_INVALID_ARG, "pool beyond 2^31 - 1 records or 2^34 leaves");
    int rc = check_canvas_args(depth, extent);
    if (rc) return rc;
    // validation: breadth-first numbering of records and leaves, depth bound, finite FP16 values
    std::vector<uint8_t> level((size_t)n_records, 0);
    int64_t next_rec = 1, next_leaf = 0;
    unsigned long long hh = 0;
    int64_t wraps[kMaxWraps] = {};
    int32_t n_wrap = 0;
    for (int64_t r = 0; r < n_records; ++r) {
        if (r >= next_rec) return fail(CANVOX_ERR_BAD_TREE, "record %lld is not referenced before it appears", (long long)r);
        for (int k = 0; k < 8; ++k) {
            const int32_t v = node_pool[8 * r + k];
            hh += elem_hash(1ull, (unsigned long long)(8 * r + k), (unsigned long long)(uint32_t)v);
            if (v > 0) {
                if (v != next_rec)
                    return fail(CANVOX_ERR_BAD_TREE, "record %lld slot %d: child %d, expected %lld (breadth-first order)",
                                (long long)r, k, v, (long long)next_rec);
                if (v >= n_records) return fail(CANVOX_ERR_BAD_TREE, "record %lld slot %d: child %d out of range", (long long)r, k, v);
                if (level[r] + 1 > depth - 1)
                    return fail(CANVOX_ERR_BAD_TREE, "record %d at level %d exceeds depth %d", v, level[r] + 1, depth);
                level[v] = (uint8_t)(level[r] + 1);
                ++next_rec;
            } else if (v < 0) {
                // leaves are numbered in breadth-first slot order; the slot holds the number modulo 2^31
                const int64_t li = -(int64_t)v - 1;
                if (li != (next_leaf & 0x7FFFFFFFll))
                    return fail(CANVOX_ERR_BAD_TREE,
                                "record %lld slot %d: leaf %lld, expected %lld (breadth-first order, modulo 2^31)",
                                (long long)r, k, (long long)li, (long long)(next_leaf & 0x7FFFFFFFll));
                if (next_leaf >= n_leaves)
                    return fail(CANVOX_ERR_BAD_TREE, "record %lld slot %d: leaf %lld out of range", (long long)r, k,
                                (long long)next_leaf);
                if (next_leaf > 0 && li == 0) wraps[n_wrap++] = 8 * r + k;  // n_leaves <= 2^34: at most 7
                ++next_leaf;
            }
        }
    }
    if (next_rec != n_records) return fail(CANVOX_ERR_BAD_TREE, "%lld records unreachable", (long long)(n_records - next_rec));
    if (next_leaf != n_leaves) return fail(CANVOX_ERR_BAD_TREE, "%lld leaves unreferenced", (long long)(n_leaves - next_leaf));
    for (int64_t i = 0; i < n_leaves; ++i) {
        const uint16_t* q = leaf_rgba + 4 * i;
        for (int c = 0; c < 4; ++c)
            if (((q[c] >> 10) & 31) == 31) return fail(CANVOX_ERR_BAD_TREE, "leaf %lld: non-finite FP16", (long long)i);
        if ((q[3] & 0x8000u) && (q[3] & 0x7FFFu)) return fail(CANVOX_ERR_BAD_TREE, "leaf %lld: negative extinction", (long long)i);
        unsigned long long val = (unsigned long long)q[0] | ((unsigned long long)q[1] << 16) |
                                 ((unsigned long long)q[2] << 32) | ((unsigned long long)q[3] << 48);
        hh += elem_hash(2ull, (unsigned long long)i, val);
    }
    rc = ensure_device();
    if (rc) return rc;
    // replace the device copy
    if ((rc = drop_canvas())) return rc;
    paint_cache_free(g.paint_cache);  // an uploaded canvas cannot be appended to
    g.paint_cache = nullptr;
    CK(cudaMalloc(&g.d_nodes, sizeof(int32_t) * 8 * (size_t)n_records), "cudaMalloc(nodes)");
    CK(cudaMalloc(&g.d_leaves, sizeof(uint2) * (size_t)(n_leaves > 0 ? n_leaves : 1)), "cudaMalloc(leaves)");
    CK(cudaMemcpy(g.d_nodes, node_pool, sizeof(int32_t) * 8 * (size_t)n_records, cudaMemcpyHostToDevice), "cudaMemcpy(nodes)");
    if (n_leaves > 0)
        CK(cudaMemcpy(g.d_leaves, leaf_rgba, sizeof(uint2) * (size_t)n_leaves, cudaMemcpyHostToDevice), "cudaMemcpy(leaves)");
    g.n_rec = n_records;
    g.n_leaf = n_leaves;
    g.depth = depth;
    g.extent = extent;
    g.n_wrap = n_wrap;
    for (int m = 0; m < kMaxWraps; ++m) g.wrap[m] = m < n_wrap ? wraps[m] : 0;
    g.host_hash = hh;
    // bit-identity of the device copy
    CK(cudaMemset(g.d_hash, 0, sizeof(unsigned long long)), "cudaMemset(hash)");
    CK(launch_hash(device_tree(), g.d_hash, 0), "hash kernel launch");
    unsigned long long dh = 0;
    CK(cudaMemcpy(&dh, g.d_hash, sizeof(dh), cudaMemcpyDeviceToHost), "cudaMemcpy(hash)");
    if (dh != hh) return fail(CANVOX_ERR_CUDA, "device copy hash %016llx differs from host %016llx", dh, hh);
    // records of each level (breadth-first order keeps each level contiguous)
    g.level_begin.assign(1, 0);
    for (int64_t lo = 0; lo < n_records;) {
        int64_t hi = lo;
        while (hi < n_records && level[(size_t)hi] == level[(size_t)lo]) ++hi;
        g.level_begin.push_back(hi);
        lo = hi;
    }
    if ((rc = build_links())) return rc;
    g.uploaded = true;
    return CANVOX_OK;
}

int canvox_paint_spheres(int32_t depth, double extent, const double* centers, const double* radii, const float* rgba,
                         int64_t n, int64_t* n_records, int64_t* n_leaves) {
    g_err.clear();
    int rc = check_stamps(centers, radii, rgba, n);
    if (rc) return rc;
    if ((rc = check_canvas_args(depth, extent))) return rc;
    if ((rc = ensure_device())) return rc;
    if ((rc = drop_canvas())) return rc;
    paint_cache_free(g.paint_cache);  // a new stamp table: painted whole
    g.paint_cache = nullptr;
    if ((rc = reserve_stamps(n, 0))) return rc;
    if (n > 0) {
        CK(cudaMemcpy(g.d_st_c, centers, sizeof(double) * 3 * (size_t)n, cudaMemcpyHostToDevice), "cudaMemcpy(stamps)");
        CK(cudaMemcpy(g.d_st_r, radii, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice), "cudaMemcpy(stamps)");
        CK(cudaMemcpy(g.d_st_rgba, rgba, sizeof(float4) * (size_t)n, cudaMemcpyHostToDevice), "cudaMemcpy(stamps)");
    }
    g.st_n = n;
    return paint_table(depth, extent, n_records, n_leaves);
}

int canvox_paint_append(const double* centers, const double* radii, const float* rgba, int64_t n, int64_t* n_records,
                        int64_t* n_leaves) {
    g_err.clear();
    if (!g.painted) return fail(CANVOX_ERR_NOT_UPLOADED, "the current canvas was not painted by canvox_paint_spheres");
    int rc = check_stamps(centers, radii, rgba, n);
    if (rc) return rc;
    if (g.st_n + n >= 0x7FFFFFFFll) return fail(CANVOX_ERR_INVALID_ARG, "stamp table beyond 2^31 - 1 stamps");
    const int32_t depth = g.depth;
    const double extent = g.extent;
    if ((rc = reserve_stamps(g.st_n + n, g.st_n))) return rc;
    if (n > 0) {
        CK(cudaMemcpy(g.d_st_c + 3 * g.st_n, centers, sizeof(double) * 3 * (size_t)n, cudaMemcpyHostToDevice),
           "cudaMemcpy(stamps)");
        CK(cudaMemcpy(g.d_st_r + g.st_n, radii, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice), "cudaMemcpy(stamps)");
        CK(cudaMemcpy(g.d_st_rgba + g.st_n, rgba, sizeof(float4) * (size_t)n, cudaMemcpyHostToDevice), "cudaMemcpy(stamps)");
    }
    if ((rc = drop_canvas())) return rc;
    g.st_n += n;
    return paint_table(depth, extent, n_records, n_leaves);
}

int canvox_canvas_info(int64_t* n_records, int64_t* n_leaves, int32_t* depth, double* extent) {
    g_err.clear();
    if (!g.uploaded) return fail(CANVOX_ERR_NOT_UPLOADED, "no canvas uploaded");
    if (n_records) *n_records = g.n_rec;
    if (n_leaves) *n_leaves = g.n_leaf;
    if (depth) *depth = g.depth;
    if (extent) *extent = g.extent;
    return CANVOX_OK;
}

int canvox_download_octree(int32_t* node_pool, uint16_t* leaf_rgba) {
    g_err.clear();
    if (!g.uploaded) return fail(CANVOX_ERR_NOT_UPLOADED, "no canvas uploaded");
    if (!node_pool || (g.n_leaf > 0 && !leaf_rgba)) return fail(CANVOX_ERR_INVALID_ARG, "null output");
    if (g.any_render) CK(cudaEventSynchronize(g.done), "cudaEventSynchronize");
    CK(cudaMemcpy(node_pool, g.d_nodes, sizeof(int32_t) * 8 * (size_t)g.n_rec, cudaMemcpyDeviceToHost), "cudaMemcpy(nodes)");
    if (g.n_leaf > 0)
        CK(cudaMemcpy(leaf_rgba, g.d_leaves, sizeof(uint2) * (size_t)g.n_leaf, cudaMemcpyDeviceToHost), "cudaMemcpy(leaves)");
    return CANVOX_OK;
}

int canvox_update_leaves(int64_t first, int64_t count, const uint16_t* leaf_rgba) {
    g_err.clear();
    if (!g.uploaded) return fail(CANVOX_ERR_NOT_UPLOADED, "no canvas uploaded");
    if (count < 0 || first < 0 || first > g.n_leaf || count > g.n_leaf - first || (count > 0 && !leaf_rgba))
        return fail(CANVOX_ERR_INVALID_ARG, "leaf range [%lld, %lld) outside the pool of %lld leaves",
                    (long long)first, (long long)(first + count), (long long)g.n_leaf);
    for (int64_t i = 0; i < count; ++i) {
        const uint16_t* q = leaf_rgba + 4 * i;
        for (int c = 0; c < 4; ++c)
            if (((q[c] >> 10) & 31) == 31) return fail(CANVOX_ERR_BAD_TREE, "leaf %lld: non-finite FP16", (long long)(first + i));
        if ((q[3] & 0x8000u) && (q[3] & 0x7FFFu))
            return fail(CANVOX_ERR_BAD_TREE, "leaf %lld: negative extinction", (long long)(first + i));
    }
    if (count == 0) return CANVOX_OK;
    if (g.any_render) CK(cudaEventSynchronize(g.done), "cudaEventSynchronize");
    // the pool hash is a sum over elements: take the old values' terms out, put the new ones in
    std::vector<uint2> old((size_t)count);
    CK(cudaMemcpy(old.data(), g.d_leaves + first, sizeof(uint2) * (size_t)count, cudaMemcpyDeviceToHost), "cudaMemcpy(leaves)");
    unsigned long long hh = g.host_hash;
    for (int64_t i = 0; i < count; ++i) {
        const uint16_t* q = leaf_rgba + 4 * i;
        const unsigned long long nv = (unsigned long long)q[0] | ((unsigned long long)q[1] << 16) |
                                      ((unsigned long long)q[2] << 32) | ((unsigned long long)q[3] << 48);
        const unsigned long long ov = ((unsigned long long)old[(size_t)i].y << 32) | old[(size_t)i].x;
        hh -= elem_hash(2ull, (unsigned long long)(first + i), ov);
        hh += elem_hash(2ull, (unsigned long long)(first + i), nv);
    }
    CK(cudaMemcpy(g.d_leaves + first, leaf_rgba, sizeof(uint2) * (size_t)count, cudaMemcpyHostToDevice), "cudaMemcpy(leaves)");
    g.host_hash = hh;
    g.last_h2d = (int64_t)sizeof(uint2) * count;
    return CANVOX_OK;
}

int canvox_octree_hash(uint64_t* host_hash, uint64_t* device_hash) {
    g_err.clear();
    if (!g.uploaded) return fail(CANVOX_ERR_NOT_UPLOADED, "no canvas uploaded");
    if (host_hash) *host_hash = g.host_hash;
    if (device_hash) {
        if (g.any_render) CK(cudaEventSynchronize(g.done), "cudaEventSynchronize");
        CK(cudaMemset(g.d_hash, 0, sizeof(unsigned long long)), "cudaMemset(hash)");
        CK(launch_hash(device_tree(), g.d_hash, 0), "hash kernel launch");
        unsigned long long dh = 0;
        CK(cudaMemcpy(&dh, g.d_hash, sizeof(dh), cudaMemcpyDeviceToHost), "cudaMemcpy(hash)");
        *device_hash = dh;
    }
    return CANVOX_OK;
}

int canvox_render_ex(const canvox_camera* cams, int32_t n_views, float* out_rgba_dev, void* stream,
                     const canvox_render_opts* opts) {
    g_err.clear();
    if (n_views < 0 || (n_views > 0 && (!cams || !out_rgba_dev))) return fail(CANVOX_ERR_INVALID_ARG, "null cameras/output or n_views < 0");
    if (!g.uploaded) return fail(CANVOX_ERR_NOT_UPLOADED, "no canvas uploaded");
    int rc = ensure_device();
    if (rc) return rc;
    canvox_render_opts o;
    rc = resolve_opts(opts, &o);
    if (rc) return rc;
    if (n_views == 0) return CANVOX_OK;
    std::vector<View> views((size_t)n_views);
    int64_t total_rays = 0;
    rc = setup_views(cams, n_views, o.tile_w, views.data(), &total_rays);
    if (rc) return rc;
    if ((rc = ensure_views(n_views)) || (rc = ensure_scratch(o.per_view ? n_views : 1))) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int b = g.next_buf;
    g.next_buf ^= 1;
    // the staging buffer b may still feed an earlier render's copy
    CK(cudaEventSynchronize(g.staged[b]), "cudaEventSynchronize(staging)");
    std::memcpy(g.h_views[b], views.data(), sizeof(View) * (size_t)n_views);
    // renders share the library's scratch: order this one after the previous one
    if (g.any_render) CK(cudaStreamWaitEvent(s, g.done, 0), "cudaStreamWaitEvent");
    if (o.use_graph) {
        unsigned long long layout = 0;
        for (int v = 0; v < n_views; ++v)
            layout = mix64(layout ^ mix64(((unsigned long long)cams[v].width << 32) ^ (unsigned long long)cams[v].height) ^
                           (unsigned long long)cams[v].out_offset_px);
        GraphEntry* hit = nullptr;
        for (auto& e : g.graphs)
            if (e.valid && e.buf == b && e.out == out_rgba_dev && e.n_views == n_views && e.total_rays == total_rays &&
                e.layout == layout && same_opts(e.opts, o))
                hit = &e;
        if (!hit) {
            GraphEntry& e = g.graphs[g.graph_next];
            g.graph_next = (g.graph_next + 1) % 4;
            if (e.exec) cudaGraphExecDestroy(e.exec);
            e = GraphEntry();
            cudaStream_t cs;
            CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "cudaStreamCreate");
            cudaGraph_t graph;
            cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (ce != cudaSuccess) {
                cudaStreamDestroy(cs);
                return cuda_fail(ce, "cudaStreamBeginCapture");
            }
            int erc = enqueue(g.h_views[b], views.data(), n_views, total_rays, out_rgba_dev, o, cs);
            ce = cudaStreamEndCapture(cs, &graph);
            cudaStreamDestroy(cs);
            if (erc) return erc;
            if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
            ce = cudaGraphInstantiate(&e.exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ce != cudaSuccess) return cuda_fail(ce, "cudaGraphInstantiate");
            e.valid = true;
            e.buf = b;
            e.out = out_rgba_dev;
            e.n_views = n_views;
            e.total_rays = total_rays;
            e.layout = layout;
            e.opts = o;
            hit = &e;
        }
        CK(cudaGraphLaunch(hit->exec, s), "cudaGraphLaunch");
    } else {
        rc = enqueue(g.h_views[b], views.data(), n_views, total_rays, out_rgba_dev, o, s);
        if (rc) return rc;
    }
    CK(cudaEventRecord(g.staged[b], s), "cudaEventRecord");
    CK(cudaEventRecord(g.done, s), "cudaEventRecord");
    g.any_render = true;
    g.last_h2d = (int64_t)sizeof(View) * n_views;
    g.last_d2h = 0;
    return CANVOX_OK;
}

int canvox_render(const canvox_camera* cams, int32_t n_views, float* out_rgba_dev, void* stream) {
    return canvox_render_ex(cams, n_views, out_rgba_dev, stream, nullptr);
}

int canvox_get_stats(canvox_stats* s) {
    g_err.clear();
    if (!s) return fail(CANVOX_ERR_INVALID_ARG, "null stats");
    std::memset(s, 0, sizeof(*s));
    if (!g.any_render) return CANVOX_OK;
    CK(cudaEventSynchronize(g.done), "cudaEventSynchronize");
    Scratch h;
    CK(cudaMemcpy(&h, g.d_scratch, sizeof(Scratch), cudaMemcpyDeviceToHost), "cudaMemcpy(stats)");
    s->rays = (int64_t)h.stats[kStatRays];
    s->steps = (int64_t)h.stats[kStatSteps];
    s->slot_reads = (int64_t)h.stats[kStatSlotReads];
    s->leaf_loads = (int64_t)h.stats[kStatLeafLoads];
    s->record_loads = (int64_t)h.stats[kStatRecordLoads];
    s->fp64_boundaries = (int64_t)h.stats[kStatFp64Boundaries];
    s->rebases = (int64_t)h.stats[kStatRebases];
    s->step_limited = (int64_t)h.stats[kStatStepLimited];
    s->h2d_bytes = g.last_h2d;
    s->d2h_bytes = g.last_d2h;
    if (h.status) return fail(CANVOX_ERR_STEP_LIMIT, "%lld rays stopped at the step limit", (long long)s->step_limited);
    return CANVOX_OK;
}

int canvox_render_host(const canvox_camera* cams, int32_t n_views, float* out_rgba_host, void* stream,
                       const canvox_render_opts* opts) {
    g_err.clear();
    if (n_views < 0 || (n_views > 0 && (!cams || !out_rgba_host))) return fail(CANVOX_ERR_INVALID_ARG, "null cameras/output");
    if (n_views == 0) return CANVOX_OK;
    int64_t npx = 0;
    for (int v = 0; v < n_views; ++v) {
        if (cams[v].width < 1 || cams[v].height < 1 || cams[v].out_offset_px < 0)
            return fail(CANVOX_ERR_INVALID_ARG, "camera %d: bad size or offset", v);
        const int64_t e = cams[v].out_offset_px + (int64_t)cams[v].width * cams[v].height;
        if (e > npx) npx = e;
    }
    if (npx > g.host_out_cap) {
        if (g.any_render) CK(cudaEventSynchronize(g.done), "cudaEventSynchronize");
        drop_graphs();
        if (g.d_host_out) cudaFree(g.d_host_out);
        g.d_host_out = nullptr;
        g.host_out_cap = 0;
        CK(cudaMalloc(&g.d_host_out, sizeof(float4) * (size_t)npx), "cudaMalloc(host render target)");
        g.host_out_cap = npx;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int rc = canvox_render_ex(cams, n_views, reinterpret_cast<float*>(g.d_host_out), stream, opts);
    if (rc) return rc;
    CK(cudaMemcpyAsync(out_rgba_host, g.d_host_out, sizeof(float4) * (size_t)npx, cudaMemcpyDeviceToHost, s),
       "cudaMemcpyAsync(image)");
    CK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    g.last_d2h = (int64_t)sizeof(float4) * npx;
    unsigned long long status = 0;
    CK(cudaMemcpy(&status, &g.d_scratch->status, sizeof(status), cudaMemcpyDeviceToHost), "cudaMemcpy(status)");
    if (status) return fail(CANVOX_ERR_STEP_LIMIT, "rays stopped at the step limit");
    return CANVOX_OK;
}

int canvox_autotune(const canvox_camera* cams, int32_t n_views, void* stream, canvox_render_opts* best) {
    g_err.clear();
    if (n_views < 1 || !cams) return fail(CANVOX_ERR_INVALID_ARG, "autotune needs at least one camera");
    if (!g.uploaded) return fail(CANVOX_ERR_NOT_UPLOADED, "no canvas uploaded");
    int64_t npx = 0;
    for (int v = 0; v < n_views; ++v) {
        const int64_t e = cams[v].out_offset_px + (int64_t)cams[v].width * cams[v].height;
        if (e > npx) npx = e;
    }
    float4* out = nullptr;
    CK(cudaMalloc(&out, sizeof(float4) * (size_t)(npx > 0 ? npx : 1)), "cudaMalloc(autotune target)");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = CANVOX_OK;
    // time one schedule: best of 2 renders after one warm-up
    auto time_opts = [&](const canvox_render_opts& o) -> float {
        float ms_min = 1e30f;
        for (int rep = 0; rep < 3 && rc == CANVOX_OK; ++rep) {
            cudaEventRecord(e0, s);
            rc = canvox_render_ex(cams, n_views, reinterpret_cast<float*>(out), stream, &o);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms < ms_min) ms_min = ms;
        }
        return ms_min;
    };
    canvox_render_opts win;
    builtin_defaults(&win);
    float best_ms = time_opts(win);
    const int blocks[] = {128, 256};
    const int refills[] = {0, 2, 4};
    const int tiles[] = {4, 8, 16, 32};
    const int smems[] = {0, 256, 1024, 4096};
    const int frames[] = {16, 20, 22};
    const int traversals[] = {0, 1};
    for (int pass = 0; pass < 2 && rc == CANVOX_OK; ++pass) {
        for (int which = 0; which < 6 && rc == CANVOX_OK; ++which) {
            const int* vals = which == 0 ? blocks : which == 1 ? refills : which == 2 ? tiles : which == 3 ? smems
                            : which == 4 ? frames : traversals;
            const int nv = which == 0 ? 2 : which == 1 ? 3 : which == 2 ? 4 : which == 3 ? 4 : which == 4 ? 3 : 2;
            for (int i = 0; i < nv && rc == CANVOX_OK; ++i) {
                canvox_render_opts o = win;
                int* field = which == 0 ? &o.block_threads : which == 1 ? &o.refill : which == 2 ? &o.tile_w
                             : which == 3 ? &o.smem_records : which == 4 ? &o.frame_levels : &o.traversal;
                if (*field == vals[i]) continue;
                *field = vals[i];
                o.blocks_per_sm = 0;
                const float ms = time_opts(o);
                if (rc == CANVOX_OK && ms < best_ms) {
                    best_ms = ms;
                    win = o;
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    cudaFree(out);
    if (rc) return rc;
    g.tuned = win;
    g.have_tuned = true;
    if (best) *best = win;
    return CANVOX_OK;
}

int canvox_footprint(const canvox_camera* cams, int32_t n_views, void* stream, int64_t* n_records, int64_t* n_leaves) {
    g_err.clear();
    if (n_views < 0 || (n_views > 0 && !cams) || !n_records || !n_leaves)
        return fail(CANVOX_ERR_INVALID_ARG, "null cameras/results or n_views < 0");
    if (!g.uploaded) return fail(CANVOX_ERR_NOT_UPLOADED, "no canvas uploaded");
    int rc = ensure_device();
    if (rc) return rc;
    canvox_render_opts o;
    builtin_defaults(&o);
    if ((rc = resolve_opts(&o, &o))) return rc;
    std::vector<View> views((size_t)(n_views > 0 ? n_views : 1));
    int64_t total_rays = 0;
    if (n_views > 0 && (rc = setup_views(cams, n_views, o.tile_w, views.data(), &total_rays))) return rc;
    if ((rc = ensure_views(n_views > 0 ? n_views : 1)) || (rc = ensure_scratch(1))) return rc;
    if (g.any_render) CK(cudaEventSynchronize(g.done), "cudaEventSynchronize");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int64_t rec_words = (g.n_rec + 31) / 32, leaf_words = (g.n_leaf + 31) / 32;
    uint32_t* bits = nullptr;
    CK(cudaMalloc(&bits, sizeof(uint32_t) * (size_t)(rec_words + leaf_words + 4)), "cudaMalloc(footprint)");
    struct Free {
        uint32_t* p;
        ~Free() { cudaFree(p); }
    } guard{bits};
    CK(cudaMemset(bits, 0, sizeof(uint32_t) * (size_t)(rec_words + leaf_words + 4)), "cudaMemset(footprint)");
    if (n_views > 0)
        CK(cudaMemcpy(g.d_views, views.data(), sizeof(View) * (size_t)n_views, cudaMemcpyHostToDevice), "cudaMemcpy(views)");
    CK(cudaMemset(g.d_scratch, 0, scratch_bytes(1)), "cudaMemset(scratch)");
    PlainParams p;
    std::memset(&p, 0, sizeof(p));
    p.tree = device_tree();
    p.scratch = g.d_scratch;
    p.step_limit = o.step_limit;
    p.t_min = o.t_min;
    p.mark_rec = bits;
    p.mark_leaf = bits + rec_words;
    for (int v = 0; v < n_views; ++v) {
        p.view = g.d_views + v;
        CK(launch_plain(p, CANVOX_PREC_FP64, (long long)views[v].width * views[v].height, s), "footprint launch");
    }
    CK(cudaStreamSynchronize(s), "cudaStreamSynchronize(footprint)");
    unsigned long long* d_count = reinterpret_cast<unsigned long long*>(bits + rec_words + leaf_words);
    if (reinterpret_cast<uintptr_t>(d_count) % 8) d_count = reinterpret_cast<unsigned long long*>(bits + rec_words + leaf_words + 1);
    CK(footprint_finish(g.d_nodes, g.level_begin.data(), (int)g.level_begin.size() - 1, bits, rec_words,
                        bits + rec_words, leaf_words, d_count, n_records, n_leaves), "footprint count");
    return CANVOX_OK;
}

int canvox_probe_l2_gather(int64_t buffer_bytes, double* sector_gbs) {
    g_err.clear();
    if (!sector_gbs || buffer_bytes < 0 || buffer_bytes > ((int64_t)1 << 36))
        return fail(CANVOX_ERR_INVALID_ARG, "buffer_bytes %lld out of range", (long long)buffer_bytes);
    int dev = 0, l2 = 0;
    CK(cudaGetDevice(&dev), "cudaGetDevice");
    if (buffer_bytes == 0) {
        CK(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev), "cudaDeviceGetAttribute(L2)");
        buffer_bytes = l2 / 2;
    }
    if (buffer_bytes < (1 << 15)) return fail(CANVOX_ERR_INVALID_ARG, "buffer_bytes below 32 KiB");
    CK(probe_l2_gather(buffer_bytes, sector_gbs), "L2 gather probe");
    return CANVOX_OK;
}

int canvox_probe_fp64(double* gflops) {
    g_err.clear();
    if (!gflops) return fail(CANVOX_ERR_INVALID_ARG, "null result");
    CK(probe_fp64(gflops), "FP64 probe");
    return CANVOX_OK;
}

void canvox_release(void) {
    if (g.device < 0) return;
    cudaDeviceSynchronize();
    drop_graphs();
    if (g.d_nodes) cudaFree(g.d_nodes);
    if (g.d_leaves) cudaFree(g.d_leaves);
    if (g.d_ropes) cudaFree(g.d_ropes);
    if (g.d_views) cudaFree(g.d_views);
    if (g.d_eye) cudaFree(g.d_eye);
    for (int b = 0; b < 2; ++b) {
        if (g.h_views[b]) cudaFreeHost(g.h_views[b]);
        if (g.staged[b]) cudaEventDestroy(g.staged[b]);
    }
    if (g.d_scratch) cudaFree(g.d_scratch);
    if (g.d_hash) cudaFree(g.d_hash);
    if (g.d_host_out) cudaFree(g.d_host_out);
    if (g.d_st_c) cudaFree(g.d_st_c);
    if (g.d_st_r) cudaFree(g.d_st_r);
    if (g.d_st_rgba) cudaFree(g.d_st_rgba);
    paint_cache_free(g.paint_cache);
    if (g.done) cudaEventDestroy(g.done);
    g = Ctx();
}

}  // extern "C"
