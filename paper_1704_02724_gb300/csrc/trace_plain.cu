// Plain single-precision-type ray casters (one launch per view), and the small
// kernels around the traversal: the pool hash, the eye leaf of each view, and
// the neighbour links built at upload.
//
// These are the baselines the mixed kernel is measured against: the ray, the
// cell planes and the compositing are all in one type R, in canvas
// coordinates, and every step locates the leaf from the root (no stack, no
// local frame). With R = double this is the plain FP64 GPU path; with
// R = float it is the canvas-coordinate FP32 traversal that Sec. 6.3 and the
// canvas-coordinate panel of its accuracy figure show drifting at depth.
// Planes are formed from integer cell coordinates, c * w_L - E/2, so a plane has
// one rounded value at every level and the located leaf always lies ahead of t.
// The FP64 caster can also mark the records and stored leaves it reads (the
// footprint of a frame, canvox_footprint).
#include <cuda_fp16.h>

#include "canvox_internal.cuh"

namespace canvox {
namespace {

template <typename R>
struct Num;
template <>
struct Num<double> {
    static __device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }
    static __device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
    static __device__ __forceinline__ double expm1_(double x) { return expm1(x); }
    static __device__ __forceinline__ double exp_(double x) { return exp(x); }
    static __device__ __forceinline__ double pow2(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }
    static __device__ __forceinline__ double inf() { return __longlong_as_double(0x7FF0000000000000ll); }
};
template <>
struct Num<float> {
    static __device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
    static __device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
    static __device__ __forceinline__ float expm1_(float x) { return expm1f(x); }
    static __device__ __forceinline__ float exp_(float x) { return expf(x); }
    static __device__ __forceinline__ float pow2(int e) { return __int_as_float((127 + e) << 23); }
    static __device__ __forceinline__ float inf() { return __int_as_float(0x7F800000); }
};

__device__ __forceinline__ float h2f(unsigned short h) { return __half2float(__ushort_as_half(h)); }

// Set bit i of a footprint bitset (read through L2 first: most bits are already set).
__device__ __forceinline__ void mark_bit(uint32_t* bits, long long i) {
    const uint32_t m = 1u << (i & 31);
    uint32_t* w = bits + (i >> 5);
    if (!(__ldcg(w) & m)) atomicOr(w, m);
}

struct PlainCount {
    unsigned long long steps, leaf_loads, rec_loads;
};

// kWrap: the canvas has more than 2^31 leaves (slots hold leaf numbers modulo 2^31); an instance
// without it reads the number straight from the slot.
template <typename R, bool kWrap>
__device__ __forceinline__ PlainCount plain_ray(const PlainParams& P, long long idx) {
    using N = Num<R>;
    const View& V = *P.view;
    const int i = (int)(idx % V.width), j = (int)(idx / V.width);
    const Tree& T = P.tree;
    const R E = (R)T.extent, half = (R)T.half;
    // pixel-centre ray: the camera model's FP64 ray, rounded to R
    R o[3], d[3], inv[3], nod[3];
    {
        double dd[3];
        pixel_ray(V, i, j, dd);
        for (int a = 0; a < 3; ++a) {
            o[a] = (R)V.eye[a];
            d[a] = (R)dd[a];
        }
    }
    R t0 = 0, t1 = N::inf();
    bool miss = false;
    for (int a = 0; a < 3; ++a) {
        if (d[a] != (R)0) {
            inv[a] = (R)1 / d[a];
            nod[a] = -o[a] * inv[a];
            const R ta = N::fma_(-half, inv[a], nod[a]), tb = N::fma_(half, inv[a], nod[a]);
            t0 = fmax(t0, d[a] > 0 ? ta : tb);
            t1 = fmin(t1, d[a] > 0 ? tb : ta);
        } else {
            inv[a] = 0;
            nod[a] = o[a];
            if (!(o[a] >= -half && o[a] < half)) miss = true;
        }
    }
    R C[3] = {0, 0, 0}, Tr = 1;
    int steps = 0;
    unsigned long long rec_loads = 0, leaf_loads = 0;
    if (!miss && t0 < t1) {
        R t = t0;
        for (;;) {
            if (steps >= P.step_limit) {
                atomicOr(&P.scratch->status, 1ull);
                atomicAdd(&P.scratch->stats[kStatStepLimited], 1ull);
                break;
            }
            // locate the leaf holding r(t+) from the root
            unsigned cc[3] = {0u, 0u, 0u};
            int lev = 0;
            int32_t rec = 0, slot;
            int64_t li = 0;  // number of the located leaf (slot < 0)
            for (;;) {
                const R w = E * N::pow2(-(lev + 1));
                int k = 0;
                for (int a = 0; a < 3; ++a) {
                    const R M = N::fma_((R)(2u * cc[a] + 1u), w, -half);
                    unsigned b;
                    if (d[a] == (R)0) {
                        b = nod[a] >= M;
                    } else {
                        const R tm = N::fma_(M, inv[a], nod[a]);
                        b = d[a] > 0 ? (tm <= t) : (tm > t);
                    }
                    cc[a] = 2u * cc[a] + b;
                    k |= (int)b << a;
                }
                slot = __ldg(T.nodes + (long long)rec * 8 + k);
                rec_loads += 1;
                if (slot > 0) {
                    rec = slot;
                    ++lev;
                } else {
                    if (slot < 0) li = kWrap ? leaf_index(T, rec, k, slot) : -(int64_t)slot - 1;
                    break;
                }
            }
            if (P.mark_rec) mark_bit(P.mark_rec, rec);
            const int L = lev + 1;
            const R w = E * N::pow2(-L);
            R te = N::inf();
            for (int a = 0; a < 3; ++a) {
                if (d[a] == (R)0) continue;
                const R F = N::fma_((R)(cc[a] + (d[a] > 0 ? 1u : 0u)), w, -half);
                const R ta = N::fma_(F, inv[a], nod[a]);
                te = fmin(te, ta);
            }
            te = fmin(te, t1);
            steps += 1;
            if (slot < 0) {
                const uint2 q = __ldg(T.leaves + li);
                leaf_loads += 1;
                if (P.mark_leaf) mark_bit(P.mark_leaf, li);
                const R s = (R)h2f((unsigned short)(q.y >> 16));
                if (s > (R)0) {
                    const R l = te - t;
                    const R a = -N::expm1_(-s * l);
                    C[0] += Tr * a * (R)h2f((unsigned short)(q.x & 0xFFFFu));
                    C[1] += Tr * a * (R)h2f((unsigned short)(q.x >> 16));
                    C[2] += Tr * a * (R)h2f((unsigned short)(q.y & 0xFFFFu));
                    Tr *= N::exp_(-s * l);
                }
            }
            if (Tr < (R)P.t_min || te >= t1) break;
            t = te;
        }
    }
    float4 out;
    out.x = (float)(C[0] + Tr * (R)V.bg[0]);
    out.y = (float)(C[1] + Tr * (R)V.bg[1]);
    out.z = (float)(C[2] + Tr * (R)V.bg[2]);
    out.w = (float)(1 - Tr);
    const long long pix = V.out_offset + idx;
    if (P.out) P.out[pix] = out;
    if (P.step_count) P.step_count[pix] = steps;
    return PlainCount{(unsigned long long)steps, leaf_loads, rec_loads};
}

template <typename R, bool kWrap>
__global__ void __launch_bounds__(256) plain_kernel(PlainParams P, long long n_pixels) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    PlainCount c = {0ull, 0ull, 0ull};
    const bool valid = idx < n_pixels;
    if (valid) c = plain_ray<R, kWrap>(P, idx);
    // counters in canvox_stats order: rays, steps, slot reads (not tracked here), leaf loads, record loads
    unsigned long long vals[5] = {valid ? 1ull : 0ull, c.steps, 0ull, c.leaf_loads, c.rec_loads};
    for (int q = 0; q < 5; ++q) {
        unsigned long long s = vals[q];
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, off);
        if ((threadIdx.x & 31) == 0 && s) atomicAdd(&P.scratch->stats[q], s);
    }
}

__global__ void hash_kernel(Tree t, unsigned long long* out) {
    unsigned long long acc = 0;
    const long long n_slots = t.n_rec * 8;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_slots; i += stride)
        acc += elem_hash(1ull, (unsigned long long)i, (unsigned long long)(uint32_t)t.nodes[i]);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < t.n_leaf; i += stride) {
        const uint2 q = t.leaves[i];
        acc += elem_hash(2ull, (unsigned long long)i, ((unsigned long long)q.y << 32) | q.x);
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

// One thread per view: the leaf holding the eye, or len = 0 when the eye is
// outside the canvas or exactly on a mid-plane of its path (then the ray's
// direction decides the side and every ray locates its own start).
__global__ void eye_path_kernel(Tree t, const View* views, int n_views, EyePath* out) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n_views) return;
    const View& V = views[v];
    EyePath& E = out[v];
    E.len = 0;
    E.stored = 0;
    E.val = make_uint2(0u, 0u);
    for (int a = 0; a < 3; ++a)
        if (!(V.eye[a] >= -t.half && V.eye[a] < t.half)) return;
    unsigned c[3] = {0u, 0u, 0u};
    int32_t rec = 0;
    for (int lev = 0; lev < kMaxDepth; ++lev) {
        E.rec[lev] = rec;
        const double w = t.extent * __longlong_as_double((long long)(1023 - (lev + 1)) << 52);
        int k = 0;
        for (int a = 0; a < 3; ++a) {
            const double M = fma((double)(2u * c[a] + 1u), w, -t.half);
            if (V.eye[a] == M) return;  // on the plane: the direction decides
            const unsigned b = V.eye[a] > M;
            c[a] = 2u * c[a] + b;
            k |= (int)b << a;
        }
        const int32_t slot = t.nodes[(long long)rec * 8 + k];
        if (slot > 0) {
            rec = slot;
            continue;
        }
        if (slot < 0) {
            E.val = t.leaves[leaf_index(t, rec, k, slot)];
            E.stored = 1;
        }
        E.c[0] = c[0];
        E.c[1] = c[1];
        E.c[2] = c[2];
        E.len = lev + 1;
        return;
    }
}

// Neighbour links (the paper's neighbour graph of Sec. 4.1.1, kept per record).
// ropes[r][2a + s] names the cell across face (axis a, s = 1 high / 0 low) of
// record r's cell: the same-level neighbour if it exists, else the coarser leaf
// that covers it, as (record holding its slot, (child index << 8) | its level);
// record -1 is outside the canvas. One launch per level, parents before
// children: a child's link is its sibling inside the parent, or the parent's
// link, refined to the adjacent child when that neighbour is an internal cell.
__global__ void rope_level_kernel(const int32_t* nodes, uint2* ropes, long long lo, long long hi, int level) {
    const long long r = lo + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= hi) return;
    if (level == 0) {
        for (int f = 0; f < 6; ++f) ropes[r * 6 + f] = make_uint2(0xFFFFFFFFu, 0u);
    }
    for (int k = 0; k < 8; ++k) {
        const int32_t v = nodes[r * 8 + k];
        if (v <= 0) continue;
        for (int f = 0; f < 6; ++f) {
            const int a = f >> 1, hi_face = f & 1;
            const int bit = (k >> a) & 1;
            const unsigned kk = (unsigned)(k ^ (1 << a));
            uint2 out;
            if (hi_face != bit) {
                out = make_uint2((unsigned)r, (kk << 8) | (unsigned)(level + 1));  // sibling inside r
            } else {
                const uint2 R = ropes[r * 6 + f];
                out = R;
                if ((int)R.x >= 0) {
                    const int32_t sv = nodes[(long long)(int)R.x * 8 + ((R.y >> 8) & 7u)];
                    if (sv > 0) out = make_uint2((unsigned)sv, (kk << 8) | (unsigned)(level + 1));
                }
            }
            ropes[(long long)v * 6 + f] = out;
        }
    }
}

}  // namespace

cudaError_t launch_rope_level(const int32_t* nodes, uint2* ropes, int64_t lo, int64_t hi, int level, cudaStream_t s) {
    if (hi <= lo) return cudaSuccess;
    const long long n = hi - lo;
    rope_level_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(nodes, ropes, lo, hi, level);
    return cudaGetLastError();
}

cudaError_t launch_eye_paths(const Tree& t, const View* views, int n_views, EyePath* out, cudaStream_t s) {
    if (n_views <= 0) return cudaSuccess;
    eye_path_kernel<<<(n_views + 63) / 64, 64, 0, s>>>(t, views, n_views, out);
    return cudaGetLastError();
}

cudaError_t launch_plain(const PlainParams& p, int precision, long long n_pixels, cudaStream_t s) {
    if (n_pixels <= 0) return cudaSuccess;
    const int block = 256;
    const long long grid = (n_pixels + block - 1) / block;
    if (grid > 0x7FFFFFFFll) return cudaErrorInvalidValue;
    const bool wrap = p.tree.n_wrap > 0;
    if (precision == CANVOX_PREC_FP32) {
        if (wrap) plain_kernel<float, true><<<(unsigned)grid, block, 0, s>>>(p, n_pixels);
        else plain_kernel<float, false><<<(unsigned)grid, block, 0, s>>>(p, n_pixels);
    } else {
        if (wrap) plain_kernel<double, true><<<(unsigned)grid, block, 0, s>>>(p, n_pixels);
        else plain_kernel<double, false><<<(unsigned)grid, block, 0, s>>>(p, n_pixels);
    }
    return cudaGetLastError();
}

cudaError_t launch_hash(const Tree& t, unsigned long long* out, cudaStream_t s) {
    hash_kernel<<<1024, 256, 0, s>>>(t, out);
    return cudaGetLastError();
}

}  // namespace canvox
