// Measurement helpers: the denominators and the footprint the traversal is
// compared with (the paper has no counterpart; it reports no profile).
//
//   canvox_probe_l2_gather : random 32-byte sector gathers from an L2-resident
//                            buffer, the access pattern of the record and leaf
//                            loads with the DRAM taken out.
//   canvox_probe_fp64      : FP64 FMA rate, the unit the plain FP64 baseline
//                            and the mixed kernel's rebases run on.
//   canvox_footprint       : the distinct records and stored leaves a render of
//                            these views reads (the compulsory bytes of a cold
//                            frame), marked by the plain FP64 traversal, which
//                            locates every leaf from the root.
#include <cstdio>
#include <vector>

#include "canvox_internal.cuh"

namespace canvox {
namespace {

constexpr int kProbeBlock = 256;
constexpr int kGatherIters = 512;  // gathers per thread (unrolled by 8)

// Each pair of lanes reads one random 32-byte sector (16 bytes each), so every
// sector fetched from L2 is used whole; loads bypass L1 (ld.global.cg).
__global__ void __launch_bounds__(kProbeBlock) gather_kernel(const uint4* __restrict__ buf, int shift,
                                                             uint32_t seed, uint32_t* sink) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t x = (tid >> 1) * 2654435761u + seed;
    const uint32_t half = tid & 1u;
    uint32_t acc = 0;
    for (int i = 0; i < kGatherIters; i += 8) {
        uint4 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            x = x * 1664525u + 1013904223u;  // LCG step (Numerical Recipes constants)
            const uint32_t sec = x >> shift;  // the top bits: a sector index below 2^(32 - shift)
            v[u] = __ldcg(buf + 2 * (size_t)sec + half);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) acc ^= v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
    }
    if (acc == 0x9E3779B9u) sink[0] = acc;  // keeps the loads; the buffer is zero, so never taken
}

constexpr int kFmaIters = 4096;

// Eight independent FP64 FMA chains per thread.
__global__ void __launch_bounds__(kProbeBlock) dfma_kernel(double seed, double* sink) {
    double a[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = seed + u + threadIdx.x;
    const double b = 0.999999, c = 1e-7;
    for (int i = 0; i < kFmaIters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = fma(a[u], b, c);
    }
    double s = 0;
#pragma unroll
    for (int u = 0; u < 8; ++u) s += a[u];
    if (s == 12345.678) sink[0] = s;
}

// Parents of marked records: one pass per level, deepest first.
__global__ void propagate_kernel(const int32_t* nodes, uint32_t* rec_bits, long long lo, long long hi) {
    const long long r = lo + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= hi) return;
    bool any = false;
    for (int k = 0; k < 8; ++k) {
        const int32_t v = nodes[r * 8 + k];
        if (v > 0 && ((rec_bits[v >> 5] >> (v & 31)) & 1u)) any = true;
    }
    if (any) atomicOr(&rec_bits[r >> 5], 1u << (r & 31));
}

__global__ void popcount_kernel(const uint32_t* bits, long long n_words, unsigned long long* out) {
    unsigned long long c = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_words; i += (long long)gridDim.x * blockDim.x)
        c += (unsigned long long)__popc(bits[i]);
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xFFFFFFFFu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

}  // namespace

cudaError_t probe_l2_gather(int64_t buffer_bytes, double* gbs) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    // a power of two of sectors, at most the requested size (2^10 .. 2^31 sectors)
    uint64_t sectors = 1ull << 10;
    int shift = 22;
    while (sectors * 2 * 32 <= (uint64_t)buffer_bytes && sectors < (1ull << 31)) {
        sectors *= 2;
        --shift;
    }
    void* buf = nullptr;
    uint32_t* sink = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    e = cudaMalloc(&buf, sectors * 32);
    if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(buf, 0, sectors * 32);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    const int grid = sms * 8;
    float best = 1e30f;
    for (int rep = 0; e == cudaSuccess && rep < 6; ++rep) {
        e = cudaEventRecord(a, 0);
        if (e != cudaSuccess) break;
        gather_kernel<<<grid, kProbeBlock>>>((const uint4*)buf, shift, 12345u + rep, sink);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(b, 0);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e == cudaSuccess && rep > 0 && ms < best) best = ms;  // the first launch warms L2
    }
    if (e == cudaSuccess) *gbs = (double)grid * kProbeBlock * kGatherIters * 16.0 / (best * 1e-3) / 1e9;
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(buf);
    cudaFree(sink);
    return e;
}

cudaError_t probe_fp64(double* gflops) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    double* sink = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    e = cudaMalloc(&sink, sizeof(double));
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    const int grid = sms * 4;
    float best = 1e30f;
    for (int rep = 0; e == cudaSuccess && rep < 4; ++rep) {
        e = cudaEventRecord(a, 0);
        if (e != cudaSuccess) break;
        dfma_kernel<<<grid, kProbeBlock>>>(1.0 + rep, sink);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(b, 0);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e == cudaSuccess && rep > 0 && ms < best) best = ms;
    }
    if (e == cudaSuccess) *gflops = 2.0 * grid * kProbeBlock * kFmaIters * 8.0 / (best * 1e-3) / 1e9;
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(sink);
    return e;
}

cudaError_t footprint_finish(const int32_t* nodes, const int64_t* level_begin, int n_levels, uint32_t* rec_bits,
                             int64_t rec_words, const uint32_t* leaf_bits, int64_t leaf_words, unsigned long long* d_count,
                             int64_t* n_records, int64_t* n_leaves) {
    // level l holds records [level_begin[l], level_begin[l + 1]); mark parents, deepest level first
    for (int l = n_levels - 1; l >= 0; --l) {
        const long long lo = level_begin[l], hi = level_begin[l + 1];
        if (hi <= lo) continue;
        propagate_kernel<<<(unsigned)((hi - lo + 255) / 256), 256>>>(nodes, rec_bits, lo, hi);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    unsigned long long c[2] = {0, 0};
    for (int w = 0; w < 2; ++w) {
        cudaError_t e = cudaMemset(d_count, 0, sizeof(unsigned long long));
        if (e != cudaSuccess) return e;
        const long long nw = w == 0 ? rec_words : leaf_words;
        if (nw > 0) {
            popcount_kernel<<<1024, 256>>>(w == 0 ? rec_bits : leaf_bits, nw, d_count);
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
        e = cudaMemcpy(&c[w], d_count, sizeof(unsigned long long), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return e;
    }
    *n_records = (int64_t)c[0];
    *n_leaves = (int64_t)c[1];
    return cudaSuccess;
}

}  // namespace canvox
