// canvox_render_noalloc: the renderer for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running inside a memory pool
// that hands out only its own blocks, a real-time loop that must not hit the
// allocator, or a host that keeps all device memory for itself. This entry
// point renders with the caller's device buffers for the octree and the image
// and keeps its own working memory (counters, ray-queue head, view table and
// per-view eye paths) in one fixed array in device global memory, declared
// below. It calls no cudaMalloc, cudaFree or other allocating routine.
#include <atomic>
#include <cmath>
#include <cstring>

#include "canvox_internal.cuh"

namespace canvox {
namespace {

constexpr int kNoallocMaxViews = 64;
constexpr size_t kOffViews = 256;  // after the Scratch header (80 bytes), 256-byte aligned
constexpr size_t kOffEye = kOffViews + ((sizeof(View) * kNoallocMaxViews + 255) / 256) * 256;
constexpr size_t kNoallocBytes = kOffEye + ((sizeof(EyePath) * kNoallocMaxViews + 255) / 256) * 256;
static_assert(sizeof(Scratch) <= kOffViews, "scratch header must fit before the view table");
static_assert(kNoallocBytes <= 24576, "the fixed scratch array is 24 KiB");

// The fixed working memory. Every GPU that loads the library holds these 24 KiB
// until the process exits. Host code must not use its name as a device address:
// it takes the address from cudaGetSymbolAddress once per device (below).
static __device__ __align__(256) unsigned char g_noalloc_scratch[24576];

// The view table of one call, passed by value as a kernel argument: the set-up kernel
// copies it into the fixed array, so no host buffer has to outlive the call.
struct ViewTable {
    View v[kNoallocMaxViews];
    int32_t n;
};
static_assert(sizeof(ViewTable) <= 32000, "kernel arguments are limited to 32764 bytes");

// Clears the counters, status word and queue head, and stores the view table.
__global__ void noalloc_setup_kernel(ViewTable t, Scratch* scratch, View* views) {
    unsigned long long* z = reinterpret_cast<unsigned long long*>(scratch);
    for (int i = threadIdx.x; i < (int)(sizeof(Scratch) / 8); i += blockDim.x) z[i] = 0ull;
    const uint32_t* src = reinterpret_cast<const uint32_t*>(t.v);
    uint32_t* dst = reinterpret_cast<uint32_t*>(views);
    const int words = t.n * (int)(sizeof(View) / 4);
    for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
}
static_assert(sizeof(Scratch) % 8 == 0 && sizeof(View) % 4 == 0, "word copies");

constexpr int kMaxDevices = 64;
// Device address of the array per device, looked up once (first call on that device). Atomic, so
// that first calls from several host threads may race on the lookup without a data race.
std::atomic<unsigned char*> g_scratch_addr[kMaxDevices];

// Device address of g_noalloc_scratch on the current device (set up on first use).
int scratch_address(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(CANVOX_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return set_error(CANVOX_ERR_INVALID_ARG, "device index out of range");
    unsigned char* a = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (!a) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return set_error(CANVOX_ERR_CUDA, cudaGetErrorString(e));
        a = static_cast<unsigned char*>(p);
        g_scratch_addr[dev].store(a, std::memory_order_release);  // every thread stores the same address
    }
    *out = a;
    return CANVOX_OK;
}

}  // namespace
}  // namespace canvox

using namespace canvox;

extern "C" int canvox_render_noalloc(const int32_t* node_pool_dev, int64_t n_records, const uint16_t* leaf_rgba_dev,
                                     int64_t n_leaves, int32_t depth, double extent, const canvox_camera* cams,
                                     int32_t n_views, float* out_rgba_dev, void* stream) {
    clear_error();
    if (n_views == 0) return CANVOX_OK;
    if (n_views < 0 || !cams || !out_rgba_dev || !node_pool_dev || n_records < 1 || n_leaves < 0 ||
        (n_leaves > 0 && !leaf_rgba_dev))
        return set_error(CANVOX_ERR_INVALID_ARG, "null pointer or bad count");
    if (n_views > kNoallocMaxViews)
        return set_error(CANVOX_ERR_INVALID_ARG, "canvox_render_noalloc takes at most 64 views per call");
    if (n_records > 0x7FFFFFFFll || n_leaves > 0x7FFFFFFFll)
        return set_error(CANVOX_ERR_INVALID_ARG, "pool larger than int32 indices");
    if (depth < 1 || depth > kMaxDepth) return set_error(CANVOX_ERR_INVALID_ARG, "depth not in 1..30");
    if (!(extent > 0.0) || !std::isfinite(extent)) return set_error(CANVOX_ERR_INVALID_ARG, "extent must be finite and > 0");
    {
        int ex;
        const double scaled = std::ldexp(std::frexp(extent, &ex), 23);
        if (scaled != std::floor(scaled)) return set_error(CANVOX_ERR_INVALID_ARG, "extent has more than 23 significant bits");
    }
    ViewTable vt;  // host stack, no heap; travels as a kernel argument
    vt.n = n_views;
    int64_t total_rays = 0;
    canvox_render_opts o;
    builtin_render_opts(&o);
    int rc = build_views(cams, n_views, o.tile_w, vt.v, &total_rays);
    if (rc) return rc;
    unsigned char* base = nullptr;
    rc = scratch_address(&base);
    if (rc) return rc;
    int dev = 0, sms = 0, bps = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = mixed_max_blocks_per_sm(o.block_threads, 0, &bps);
    if (e != cudaSuccess) return set_error(CANVOX_ERR_CUDA, cudaGetErrorString(e));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Scratch* scratch = reinterpret_cast<Scratch*>(base);
    View* views = reinterpret_cast<View*>(base + kOffViews);
    EyePath* eye = reinterpret_cast<EyePath*>(base + kOffEye);
    // the array keeps the previous call's contents: the counters and queue head start at zero
    noalloc_setup_kernel<<<1, 256, 0, s>>>(vt, scratch, views);
    e = cudaGetLastError();
    Tree t;
    t.nodes = node_pool_dev;
    t.ropes = nullptr;
    t.leaves = reinterpret_cast<const uint2*>(leaf_rgba_dev);
    t.n_rec = n_records;
    t.n_leaf = n_leaves;
    t.depth = depth;
    t.n_wrap = 0;  // n_leaves < 2^31: no leaf number passes 2^31
    t.extent = extent;
    t.half = 0.5 * extent;
    if (e == cudaSuccess) e = launch_eye_paths(t, views, n_views, eye, s);
    if (e != cudaSuccess) return set_error(CANVOX_ERR_CUDA, cudaGetErrorString(e));
    MixedParams p;
    std::memset(&p, 0, sizeof(p));
    p.tree = t;
    p.views = views;
    p.eye = eye;
    p.n_views = n_views;
    p.refill = o.refill;
    p.total_rays = total_rays;
    p.ray_base = 0;
    p.out = reinterpret_cast<float4*>(out_rgba_dev);
    p.step_count = nullptr;
    p.queue = scratch->queue;
    p.scratch = scratch;
    const int64_t lim = 3 * ((int64_t)1 << depth) + 8;
    p.step_limit = lim > 0x7FFFFFFF ? 0x7FFFFFFF : lim;
    p.t_min = 9.5367431640625e-07f;  // 2^-20
    p.err_budget = o.err_budget;
    p.frame_levels = o.frame_levels;
    p.smem_records = 0;
    p.use_ropes = 0;  // no neighbour links without allocating them
    p.count_reads = 0;  // these calls report no counters
    e = launch_mixed(p, sms * (bps > 0 ? bps : 1), o.block_threads, s);
    if (e != cudaSuccess) return set_error(CANVOX_ERR_CUDA, cudaGetErrorString(e));
    return CANVOX_OK;
}
