// Device-side stamp painter: spherical brush stamps -> canonical octree pools on the GPU.
//
// The brush model of Sec. 5: a stamp refines every cell it partially covers
// down to its target depth (the smallest k with E 2^-k <= r/10, about ten
// cells across the radius, Sec. 5.2), paints cells that lie inside the sphere
// whole, and paints the finest partially covered cells by their centre; a
// cell that is already refined when the stamp arrives is descended instead.
// Paint values are blended additively (Sec. 5.1): rgb' = B m + (1-m) C with
// m = B_a / (B_a + C_a), a' = B_a + C_a, in FP32 with every operation rounded
// separately. Leaves are then rounded to FP16, eight identical siblings merge
// into one leaf, and the pools are written in breadth-first order (Sec. 4.1.1:
// eight children per allocation unit, index-based pools).
//
// The stamps are applied in order, but the result has a closed form that is
// computed level by level without replaying them:
//   * cell C is refined iff some stamp partially covers it and has its target
//     depth below C (firstref(C) = the first such stamp, else none);
//   * a stamp s descends through C iff C is refined by the time s arrives,
//     i.e. firstref(C) <= s;
//   * a leaf's value is the blend, in stamp order, of the stamps that paint
//     it: s paints leaf X when, walking down X's ancestors from the root, the
//     first cell s does not descend through lies inside s, or is partially
//     covered and has its centre inside s.
// Each level keeps, per refined cell, the ordered list of stamps that still
// descend (undecided) or already paint its whole subtree (painted); a child
// (one warp) classifies its parent's list against its own box, 32 entries at
// a time, so a cell around a room with tens of thousands of stamps is split
// across lanes instead of one thread. Geometry is FP64 with the
// same operations and order as the host painter, so the pools are identical.
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_fp16.h>

#include "canvox_internal.cuh"

namespace canvox {
namespace {

constexpr uint64_t kInternal = 1ull << 63;  // child slot: internal cell, low bits = index at the next level
constexpr uint64_t kNotCollapsed = 1ull << 63;

struct StampDev {
    const double* c;     // [n][3]
    const double* r2;    // [n]
    const int32_t* kt;   // [n] target depth
    const float4* rgba;  // [n]
};

__device__ __forceinline__ double sq(double x) { return __dmul_rn(x, x); }

// Squared distances from the sphere centre to the box [lo, lo + h]^3 and to its farthest corner.
__device__ __forceinline__ void box_dist2(const double* c, const double lo[3], double h, double& dmin2, double& dmax2) {
    dmin2 = 0.0;
    dmax2 = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double l = lo[a], u = __dadd_rn(lo[a], h);
        if (c[a] < l) dmin2 = __dadd_rn(dmin2, sq(__dsub_rn(l, c[a])));
        else if (c[a] > u) dmin2 = __dadd_rn(dmin2, sq(__dsub_rn(c[a], u)));
        dmax2 = __dadd_rn(dmax2, fmax(sq(__dsub_rn(c[a], l)), sq(__dsub_rn(u, c[a]))));
    }
}

__device__ __forceinline__ void blend(float4& C, float4 B) {
    const float s = __fadd_rn(B.w, C.w);
    if (s == 0.0f) return;
    const float m = __fdiv_rn(B.w, s);
    const float om = __fsub_rn(1.0f, m);
    C.x = __fadd_rn(__fmul_rn(B.x, m), __fmul_rn(om, C.x));
    C.y = __fadd_rn(__fmul_rn(B.y, m), __fmul_rn(om, C.y));
    C.z = __fadd_rn(__fmul_rn(B.z, m), __fmul_rn(om, C.z));
    C.w = s;
}

// FP16 leaf key (R | G << 16 | B << 32 | sigma << 48), 0 when sigma rounds to zero.
__device__ __forceinline__ uint64_t leaf_key(float4 v) {
    const float r = fminf(fmaxf(v.x, 0.0f), 1.0f), g = fminf(fmaxf(v.y, 0.0f), 1.0f), b = fminf(fmaxf(v.z, 0.0f), 1.0f);
    const float a = fminf(fmaxf(v.w, 0.0f), 60000.0f);
    const uint64_t ha = __half_as_ushort(__float2half_rn(a));
    if (ha == 0) return 0;
    return (uint64_t)__half_as_ushort(__float2half_rn(r)) | ((uint64_t)__half_as_ushort(__float2half_rn(g)) << 16) |
           ((uint64_t)__half_as_ushort(__float2half_rn(b)) << 32) | (ha << 48);
}

struct LevelIn {
    int64_t n;              // refined cells at this level
    int32_t level;
    const uint32_t* coord;  // [n][3]
    const int64_t* off;     // [n + 1]
    const int32_t* ent;     // s: descends, ~s: paints the whole cell
};

// Box of child k of cell i at level l + 1.
__device__ __forceinline__ void child_box(const LevelIn& L, int64_t i, int k, double extent, double half, uint32_t cc[3],
                                          double lo[3], double& h) {
    h = extent * __longlong_as_double((long long)(1023 - (L.level + 1)) << 52);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        cc[a] = 2u * L.coord[3 * i + a] + ((k >> a) & 1u);
        lo[a] = fma((double)cc[a], h, -half);  // exact: a multiple of h inside the canvas
    }
}

enum { kDrop = 0, kPaint = 1, kKeep = 2 };

// Classify stamp s (undecided at the parent) for a child box; refined = child refined by the time s arrives.
__device__ __forceinline__ int classify(const StampDev& S, int32_t s, const double lo[3], double h, bool refined) {
    double dmin2, dmax2;
    const double r2 = S.r2[s];
    box_dist2(S.c + 3 * (int64_t)s, lo, h, dmin2, dmax2);
    if (dmin2 >= r2) return kDrop;
    if (dmax2 <= r2) return kPaint;
    if (refined) return kKeep;
    const double hh = 0.5 * h;
    const double* c = S.c + 3 * (int64_t)s;
    const double d2 = __dadd_rn(__dadd_rn(sq(__dsub_rn(__dadd_rn(lo[0], hh), c[0])), sq(__dsub_rn(__dadd_rn(lo[1], hh), c[1]))),
                                sq(__dsub_rn(__dadd_rn(lo[2], hh), c[2])));
    return d2 < r2 ? kPaint : kDrop;
}

// One warp per child; lanes take the parent's list 32 entries at a time, in order.
constexpr unsigned kFullMask = 0xFFFFFFFFu;
constexpr int kWarpsPerBlock = 4;

// First stamp of the list that refines the child (partially covers it, target depth below it).
__device__ __forceinline__ int32_t first_refining(const LevelIn& L, const StampDev& S, int64_t b, int64_t e, int lc,
                                                  int32_t depth, const double lo[3], double h, int lane) {
    if (lc >= depth) return 0x7FFFFFFF;
    for (int64_t base = b; base < e; base += 32) {
        const int64_t q = base + lane;
        int32_t v = -1;
        bool qual = false;
        if (q < e) {
            v = L.ent[q];
            if (v >= 0 && S.kt[v] > lc) {
                double dmin2, dmax2;
                box_dist2(S.c + 3 * (int64_t)v, lo, h, dmin2, dmax2);
                const double r2 = S.r2[v];
                qual = dmin2 < r2 && dmax2 > r2;
            }
        }
        const unsigned m = __ballot_sync(kFullMask, qual);
        if (m) return __shfl_sync(kFullMask, v, __ffs(m) - 1);  // entries are in stamp order
    }
    return 0x7FFFFFFF;
}

// The child's first refining stamp, then either its leaf key or the size of its list.
__global__ void __launch_bounds__(32 * kWarpsPerBlock) expand_count(LevelIn L, StampDev S, int32_t depth, double extent,
                                                                    double half, int32_t* firstref, uint64_t* slot,
                                                                    int64_t* count, int64_t* is_int) {
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= 8 * L.n) return;  // warp-uniform
    const int64_t i = t >> 3;
    const int k = (int)(t & 7);
    uint32_t cc[3];
    double lo[3], h;
    child_box(L, i, k, extent, half, cc, lo, h);
    const int lc = L.level + 1;
    const int64_t b = L.off[i], e = L.off[i + 1];
    const int32_t fr = first_refining(L, S, b, e, lc, depth, lo, h, lane);
    if (fr != 0x7FFFFFFF) {
        int64_t n = 0;
        for (int64_t base = b; base < e; base += 32) {
            const int64_t q = base + lane;
            bool keep = false;
            if (q < e) {
                const int32_t v = L.ent[q];
                keep = v < 0 || classify(S, v, lo, h, fr <= v) != kDrop;
            }
            n += __popc(__ballot_sync(kFullMask, keep));
        }
        if (lane == 0) {
            firstref[t] = fr;
            count[t] = n;
            is_int[t] = 1;
            slot[t] = kInternal;
        }
    } else {
        // a leaf: blend the stamps that paint it, in stamp order (every lane folds the same sequence)
        float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int64_t base = b; base < e; base += 32) {
            const int64_t q = base + lane;
            bool paint = false;
            int32_t s = 0;
            if (q < e) {
                const int32_t v = L.ent[q];
                s = v < 0 ? ~v : v;
                paint = v < 0 || classify(S, v, lo, h, false) == kPaint;
            }
            unsigned m = __ballot_sync(kFullMask, paint);
            while (m) {
                const int j = __ffs(m) - 1;
                m &= m - 1;
                blend(val, S.rgba[__shfl_sync(kFullMask, s, j)]);
            }
        }
        if (lane == 0) {
            firstref[t] = fr;
            count[t] = 0;
            is_int[t] = 0;
            slot[t] = leaf_key(val);
        }
    }
}

// Refined children: coordinates, list offsets and entries at the next level, slot = index there.
__global__ void __launch_bounds__(32 * kWarpsPerBlock) expand_write(LevelIn L, StampDev S, double extent, double half,
                                                                    const int32_t* firstref, uint64_t* slot,
                                                                    const int64_t* ent_off, const int64_t* next_idx,
                                                                    uint32_t* ncoord, int64_t* noff, int32_t* nent) {
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= 8 * L.n) return;
    if (slot[t] != kInternal) return;  // warp-uniform
    const int64_t i = t >> 3;
    const int k = (int)(t & 7);
    uint32_t cc[3];
    double lo[3], h;
    child_box(L, i, k, extent, half, cc, lo, h);
    const int32_t fr = firstref[t];
    const int64_t j = next_idx[t];
    int64_t w = ent_off[t];
    __syncwarp();
    if (lane == 0) {
        slot[t] = kInternal | (uint64_t)j;
        ncoord[3 * j] = cc[0];
        ncoord[3 * j + 1] = cc[1];
        ncoord[3 * j + 2] = cc[2];
        noff[j] = w;
    }
    const int64_t b = L.off[i], e = L.off[i + 1];
    for (int64_t base = b; base < e; base += 32) {
        const int64_t q = base + lane;
        int32_t out = 0;
        bool keep = false;
        if (q < e) {
            const int32_t v = L.ent[q];
            if (v < 0) {
                out = v;
                keep = true;
            } else {
                const int c = classify(S, v, lo, h, fr <= v);
                keep = c != kDrop;
                out = c == kPaint ? ~v : v;
            }
        }
        const unsigned m = __ballot_sync(kFullMask, keep);
        if (keep) nent[w + __popc(m & ((1u << lane) - 1u))] = out;
        w += __popc(m);
    }
}

// Stamps that touch the canvas, in order (the root's list).
__global__ void root_flags(StampDev S, int64_t n, double extent, double half, int64_t* flag) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const double lo[3] = {-half, -half, -half};
    double dmin2, dmax2;
    box_dist2(S.c + 3 * s, lo, extent, dmin2, dmax2);
    flag[s] = dmin2 < S.r2[s] ? 1 : 0;
}
__global__ void root_write(int64_t n, const int64_t* flag_scan, const int64_t* flag, int32_t* ent) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n && flag[s]) ent[flag_scan[s]] = (int32_t)s;
}

// Merge of identical siblings, bottom-up: ckey = the common key of a cell's eight children, else kNotCollapsed.
__global__ void collapse_level(int64_t n, const uint64_t* slot, const uint64_t* ckey_next, uint64_t* ckey, bool is_root) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t k0 = 0;
    bool same = !is_root;
    for (int k = 0; k < 8 && same; ++k) {
        const uint64_t v = slot[8 * i + k];
        const uint64_t key = (v & kInternal) ? ckey_next[v & ~kInternal] : v;
        if (key == kNotCollapsed) same = false;
        else if (k == 0) k0 = key;
        else if (key != k0) same = false;
    }
    ckey[i] = same ? k0 : kNotCollapsed;
}

// Surviving records and their stored-leaf counts.
__global__ void survive_count(int64_t n, const uint64_t* slot, const uint64_t* ckey_next, const uint64_t* ckey,
                              int64_t* surv, int64_t* nleaf) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bool s = ckey[i] == kNotCollapsed;
    int64_t c = 0;
    if (s) {
        for (int k = 0; k < 8; ++k) {
            const uint64_t v = slot[8 * i + k];
            const uint64_t key = (v & kInternal) ? ckey_next[v & ~kInternal] : v;
            if (key != kNotCollapsed && key != 0) ++c;
        }
    }
    surv[i] = s ? 1 : 0;
    nleaf[i] = c;
}

// Pool rows of the surviving records of one level.
__global__ void write_level(int64_t n, const uint64_t* slot, const uint64_t* ckey_next, const int64_t* rec_scan,
                            const int64_t* leaf_scan, const int64_t* surv, int64_t rec_base, int64_t next_rec_base,
                            int64_t leaf_base, const int64_t* next_rec_scan, int32_t* nodes, uint2* leaves) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !surv[i]) return;
    const int64_t r = rec_base + rec_scan[i];
    int64_t lf = leaf_base + leaf_scan[i];
    for (int k = 0; k < 8; ++k) {
        const uint64_t v = slot[8 * i + k];
        int32_t out;
        uint64_t key;
        if ((v & kInternal) && ckey_next[v & ~kInternal] == kNotCollapsed) {
            out = (int32_t)(next_rec_base + next_rec_scan[v & ~kInternal]);
        } else {
            key = (v & kInternal) ? ckey_next[v & ~kInternal] : v;
            if (key == 0) {
                out = 0;
            } else {
                leaves[lf] = make_uint2((uint32_t)key, (uint32_t)(key >> 32));
                out = -(int32_t)lf - 1;
                ++lf;
            }
        }
        nodes[8 * r + k] = out;
    }
}

// In-place exclusive scan of int64 (three phases; block sums scanned recursively).
constexpr int kScanBlock = 1024;
__global__ void scan_block(int64_t* d, int64_t n, int64_t* sums) {
    __shared__ int64_t s[kScanBlock];
    const int64_t g = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    const int64_t x = g < n ? d[g] : 0;
    s[threadIdx.x] = x;
    __syncthreads();
    for (int o = 1; o < kScanBlock; o <<= 1) {
        const int64_t y = threadIdx.x >= (unsigned)o ? s[threadIdx.x - o] : 0;
        __syncthreads();
        s[threadIdx.x] += y;
        __syncthreads();
    }
    if (g < n) d[g] = s[threadIdx.x] - x;
    if (threadIdx.x == kScanBlock - 1) sums[blockIdx.x] = s[threadIdx.x];
}
__global__ void scan_add(int64_t* d, int64_t n, const int64_t* sums) {
    const int64_t g = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    if (g < n) d[g] += sums[blockIdx.x];
}

}  // namespace

// Exclusive scan of d[0..n) in place; returns the total through *total (synchronous).
cudaError_t scan_i64(int64_t* d, int64_t n, int64_t* total) {
    if (n <= 0) {
        *total = 0;
        return cudaSuccess;
    }
    const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    int64_t* sums = nullptr;
    cudaError_t e = cudaMalloc(&sums, sizeof(int64_t) * (size_t)(nb + 1));
    if (e != cudaSuccess) return e;
    scan_block<<<(unsigned)nb, kScanBlock>>>(d, n, sums);
    e = cudaGetLastError();
    int64_t t = 0;
    if (e == cudaSuccess) {
        if (nb > 1) {
            e = scan_i64(sums, nb, &t);  // sums becomes the block offsets
            if (e == cudaSuccess) {
                scan_add<<<(unsigned)nb, kScanBlock>>>(d, n, sums);
                e = cudaGetLastError();
            }
        } else {
            e = cudaMemcpy(&t, sums, sizeof(int64_t), cudaMemcpyDeviceToHost);
        }
    }
    cudaFree(sums);
    *total = t;
    return e;
}

namespace {

struct DevBuf {
    std::vector<void*> ptrs;
    ~DevBuf() {
        for (void* p : ptrs) cudaFree(p);
    }
    template <typename T>
    cudaError_t alloc(T** p, int64_t n) {
        *p = nullptr;
        cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (size_t)(n > 0 ? n : 1));
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
    void release(void* p) {
        for (auto& q : ptrs)
            if (q == p) {
                cudaFree(q);
                q = nullptr;
            }
    }
};

unsigned blocks_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

#define PCK(call)                                    \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return e_;            \
    } while (0)

cudaError_t paint_pools(int32_t depth, double extent, const double* h_centers, const double* h_radii, const float* h_rgba,
                        int64_t n, int32_t** d_nodes_out, uint2** d_leaves_out, int64_t* n_rec_out, int64_t* n_leaf_out,
                        std::vector<int64_t>* level_begin) {
    const double half = 0.5 * extent;
    DevBuf buf;
    // stamps: centres, squared radii, target depths (host integer loop, as the host painter), colours
    std::vector<double> r2((size_t)(n > 0 ? n : 1));
    std::vector<int32_t> kt((size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
        r2[(size_t)i] = h_radii[i] * h_radii[i];
        int32_t k = 0;
        double w = extent;
        const double tgt = h_radii[i] / 10.0;
        while (k < depth && w > tgt) {
            w *= 0.5;
            ++k;
        }
        kt[(size_t)i] = k;
    }
    double *d_c, *d_r2;
    int32_t* d_kt;
    float4* d_rgba;
    PCK(buf.alloc(&d_c, 3 * n));
    PCK(buf.alloc(&d_r2, n));
    PCK(buf.alloc(&d_kt, n));
    PCK(buf.alloc(&d_rgba, n));
    if (n > 0) {
        PCK(cudaMemcpy(d_c, h_centers, sizeof(double) * 3 * (size_t)n, cudaMemcpyHostToDevice));
        PCK(cudaMemcpy(d_r2, r2.data(), sizeof(double) * (size_t)n, cudaMemcpyHostToDevice));
        PCK(cudaMemcpy(d_kt, kt.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice));
        PCK(cudaMemcpy(d_rgba, h_rgba, sizeof(float4) * (size_t)n, cudaMemcpyHostToDevice));
    }
    const StampDev S{d_c, d_r2, d_kt, d_rgba};
    // level 0: the root and the stamps that touch the canvas
    int64_t *flag, n_root = 0;
    PCK(buf.alloc(&flag, n));
    if (n > 0) {
        root_flags<<<blocks_for(n, 256), 256>>>(S, n, extent, half, flag);
        PCK(cudaGetLastError());
    }
    int64_t* flag_scan;
    PCK(buf.alloc(&flag_scan, n));
    if (n > 0) {
        PCK(cudaMemcpy(flag_scan, flag, sizeof(int64_t) * (size_t)n, cudaMemcpyDeviceToDevice));
        PCK(scan_i64(flag_scan, n, &n_root));
    }
    uint32_t* coord;
    int64_t* off;
    int32_t* ent;
    PCK(buf.alloc(&coord, 3));
    PCK(buf.alloc(&off, 2));
    PCK(buf.alloc(&ent, n_root));
    PCK(cudaMemset(coord, 0, 3 * sizeof(uint32_t)));
    const int64_t off0[2] = {0, n_root};
    PCK(cudaMemcpy(off, off0, sizeof(off0), cudaMemcpyHostToDevice));
    if (n > 0) {
        root_write<<<blocks_for(n, 256), 256>>>(n, flag_scan, flag, ent);
        PCK(cudaGetLastError());
    }
    buf.release(flag);
    buf.release(flag_scan);
    // top-down: refined cells level by level, child slots kept for the output
    std::vector<uint64_t*> slots;
    std::vector<int64_t> ncell;
    LevelIn L{1, 0, coord, off, ent};
    for (;;) {
        const int64_t nch = 8 * L.n;
        int32_t* fr;
        uint64_t* slot;
        int64_t *cnt, *isint;
        PCK(buf.alloc(&fr, nch));
        PCK(buf.alloc(&slot, nch));
        PCK(buf.alloc(&cnt, nch));
        PCK(buf.alloc(&isint, nch));
        expand_count<<<blocks_for(nch, kWarpsPerBlock), 32 * kWarpsPerBlock>>>(L, S, depth, extent, half, fr, slot, cnt,
                                                                                   isint);
        PCK(cudaGetLastError());
        int64_t n_ent = 0, n_next = 0;
        PCK(scan_i64(cnt, nch, &n_ent));
        PCK(scan_i64(isint, nch, &n_next));
        slots.push_back(slot);
        ncell.push_back(L.n);
        if (n_next == 0) {
            buf.release(fr);
            buf.release(cnt);
            buf.release(isint);
            break;
        }
        uint32_t* ncoord;
        int64_t* noff;
        int32_t* nent;
        PCK(buf.alloc(&ncoord, 3 * n_next));
        PCK(buf.alloc(&noff, n_next + 1));
        PCK(buf.alloc(&nent, n_ent));
        PCK(cudaMemcpy(noff + n_next, &n_ent, sizeof(int64_t), cudaMemcpyHostToDevice));
        expand_write<<<blocks_for(nch, kWarpsPerBlock), 32 * kWarpsPerBlock>>>(L, S, extent, half, fr, slot, cnt, isint,
                                                                                   ncoord, noff, nent);
        PCK(cudaGetLastError());
        PCK(cudaDeviceSynchronize());
        buf.release(fr);
        buf.release(cnt);
        buf.release(isint);
        buf.release(const_cast<uint32_t*>(L.coord));
        buf.release(const_cast<int64_t*>(L.off));
        buf.release(const_cast<int32_t*>(L.ent));
        L = LevelIn{n_next, L.level + 1, ncoord, noff, nent};
    }
    buf.release(const_cast<uint32_t*>(L.coord));
    buf.release(const_cast<int64_t*>(L.off));
    buf.release(const_cast<int32_t*>(L.ent));
    // bottom-up merge of identical siblings
    const int nl = (int)slots.size();
    std::vector<uint64_t*> ckey((size_t)nl + 1, nullptr);
    uint64_t* none;  // below the deepest level: no refined cells
    PCK(buf.alloc(&none, 1));
    ckey[(size_t)nl] = none;
    for (int l = nl - 1; l >= 0; --l) {
        PCK(buf.alloc(&ckey[(size_t)l], ncell[(size_t)l]));
        collapse_level<<<blocks_for(ncell[(size_t)l], 256), 256>>>(ncell[(size_t)l], slots[(size_t)l], ckey[(size_t)l + 1],
                                                                  ckey[(size_t)l], l == 0);
        PCK(cudaGetLastError());
    }
    // breadth-first numbering: records level by level, leaves in slot order
    std::vector<int64_t*> rec_scan((size_t)nl + 1, nullptr), leaf_scan((size_t)nl, nullptr), surv((size_t)nl, nullptr);
    std::vector<int64_t> rec_base((size_t)nl + 1, 0), leaf_base((size_t)nl + 1, 0);
    for (int l = 0; l < nl; ++l) {
        const int64_t nc = ncell[(size_t)l];
        PCK(buf.alloc(&surv[(size_t)l], nc));
        PCK(buf.alloc(&rec_scan[(size_t)l], nc));
        PCK(buf.alloc(&leaf_scan[(size_t)l], nc));
        survive_count<<<blocks_for(nc, 256), 256>>>(nc, slots[(size_t)l], ckey[(size_t)l + 1], ckey[(size_t)l],
                                                     rec_scan[(size_t)l], leaf_scan[(size_t)l]);
        PCK(cudaGetLastError());
        PCK(cudaMemcpy(surv[(size_t)l], rec_scan[(size_t)l], sizeof(int64_t) * (size_t)nc, cudaMemcpyDeviceToDevice));
        int64_t nr = 0, nlf = 0;
        PCK(scan_i64(rec_scan[(size_t)l], nc, &nr));
        PCK(scan_i64(leaf_scan[(size_t)l], nc, &nlf));
        rec_base[(size_t)l + 1] = rec_base[(size_t)l] + nr;
        leaf_base[(size_t)l + 1] = leaf_base[(size_t)l] + nlf;
    }
    const int64_t n_rec = rec_base[(size_t)nl], n_leaf = leaf_base[(size_t)nl];
    int32_t* d_nodes = nullptr;
    uint2* d_leaves = nullptr;
    PCK(cudaMalloc(&d_nodes, sizeof(int32_t) * 8 * (size_t)n_rec));
    cudaError_t e = cudaMalloc(&d_leaves, sizeof(uint2) * (size_t)(n_leaf > 0 ? n_leaf : 1));
    if (e != cudaSuccess) {
        cudaFree(d_nodes);
        return e;
    }
    int64_t* zero_scan;
    PCK(buf.alloc(&zero_scan, 1));
    for (int l = 0; l < nl && e == cudaSuccess; ++l) {
        const int64_t nc = ncell[(size_t)l];
        write_level<<<blocks_for(nc, 256), 256>>>(nc, slots[(size_t)l], ckey[(size_t)l + 1], rec_scan[(size_t)l],
                                                   leaf_scan[(size_t)l], surv[(size_t)l], rec_base[(size_t)l],
                                                   rec_base[(size_t)l + 1], leaf_base[(size_t)l],
                                                   l + 1 < nl ? rec_scan[(size_t)l + 1] : zero_scan, d_nodes, d_leaves);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(d_nodes);
        cudaFree(d_leaves);
        return e;
    }
    *d_nodes_out = d_nodes;
    *d_leaves_out = d_leaves;
    *n_rec_out = n_rec;
    *n_leaf_out = n_leaf;
    level_begin->clear();
    for (int l = 0; l <= nl; ++l)
        if (l == 0 || rec_base[(size_t)l] > rec_base[(size_t)l - 1]) level_begin->push_back(rec_base[(size_t)l]);
    return cudaSuccess;
}

}  // namespace canvox
