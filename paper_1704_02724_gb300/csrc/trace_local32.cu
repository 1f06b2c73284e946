// The paper's single-precision traversals, for its precision experiment (Sec. 6.2-6.3).
//
// Cell-local (CANVOX_PREC_CELL32): the ray's entry point p lives in the frame
// of the current cell (origin at the cell centre, unit size, p in [-0.5, 0.5]);
// the exit is t = (+-0.5 - p_a) / d_a on the nearest face, the exit point
// p' = p + t d, and the entry point in the next cell is p' s + c (s the ratio of
// cell sizes, c the offset of the centres). Every step rounds in FP32, so the
// position drifts by at most about 2.5 eps of the cell per step: e0 + 7.5 eps L
// over a ray of length L, an angle of at most asin(sqrt(2) (e0/L + 7.5 eps)).
//
// Canvas coordinates (CANVOX_PREC_WORLD32): the same walk with p in FP32 canvas
// coordinates and cell planes rounded to FP32 (the paper's "canvas coordinate"
// comparison); the drift then scales with the coordinates, not the cells.
//
// Cell-local in half precision (CANVOX_PREC_CELL16): the cell-local walk with
// every geometric quantity (p, d, t, p', the scale and offset) in IEEE binary16,
// eps = 2^-10; the section closes by noting that the cell-local frame would let
// a half-precision GPU trace the canvas. Compositing stays in FP32.
//
// All three write, per pixel and on request, the angle between the initial ray
// direction and the line from the eye to the ray's final position (degrees).
// The eye and the pixel ray are the FP64 camera model; the start leaf is
// located in FP64 as in the other kernels; leaves are located from the root
// each step from integer coordinates, and by the FP32 position below the
// level of the cell the ray leaves.
#include <cuda_fp16.h>

#include "canvox_internal.cuh"

namespace canvox {
namespace {

__device__ __forceinline__ float h2f32(unsigned short h) {
    const float m = __int_as_float((int)((h & 0x7FFFu) << 13)) * 5.192296858534828e+33f;  // * 2^112
    return __int_as_float(__float_as_int(m) | (int)((h & 0x8000u) << 16));
}
__device__ __forceinline__ double p2d(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }

// Geometry arithmetic of a walk: FP32 or binary16, every operation rounded to nearest.
struct Geo32 {
    using T = float;
    static __device__ __forceinline__ T from_d(double x) { return (float)x; }
    static __device__ __forceinline__ T from_f(float x) { return x; }
    static __device__ __forceinline__ float f(T x) { return x; }
    static __device__ __forceinline__ T add(T a, T b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ T sub(T a, T b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ T mul(T a, T b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ T div(T a, T b) { return __fdiv_rn(a, b); }
};
struct Geo16 {
    using T = __half;
    static __device__ __forceinline__ T from_d(double x) { return __double2half(x); }
    static __device__ __forceinline__ T from_f(float x) { return __float2half_rn(x); }
    static __device__ __forceinline__ float f(T x) { return __half2float(x); }
    static __device__ __forceinline__ T add(T a, T b) { return __hadd(a, b); }
    static __device__ __forceinline__ T sub(T a, T b) { return __hsub(a, b); }
    static __device__ __forceinline__ T mul(T a, T b) { return __hmul(a, b); }
    static __device__ __forceinline__ T div(T a, T b) { return __hdiv(a, b); }
};

struct Local32Count {
    unsigned long long steps, leaf_loads, rec_loads;
};

// Leaf slot holding the cell (L, c) or its coarsest ancestor leaf; returns the slot and the leaf level.
__device__ __forceinline__ int32_t locate_int(const Tree& T, const unsigned c[3], int L, int* Lleaf, int32_t* rec_out,
                                              int* k_out, unsigned long long* loads) {
    int32_t rec = 0;
    for (int lev = 0;; ++lev) {
        const int sh = L - 1 - lev;
        const int k = (int)((c[0] >> sh) & 1u) | (int)(((c[1] >> sh) & 1u) << 1) | (int)(((c[2] >> sh) & 1u) << 2);
        const int32_t slot = __ldg(T.nodes + (long long)rec * 8 + k);
        *loads += 1;
        if (slot <= 0 || lev + 1 == L) {
            *Lleaf = lev + 1;
            *rec_out = rec;
            *k_out = k;
            return slot;
        }
        rec = slot;
    }
}

template <bool kCellLocal, typename G>
__device__ Local32Count local32_ray(const PlainParams& P, long long idx) {
    using GT = typename G::T;
    const View& V = *P.view;
    const Tree& T = P.tree;
    const int i = (int)(idx % V.width), j = (int)(idx / V.width);
    double d64[3];
    pixel_ray(V, i, j, d64);
    const double* o = V.eye;
    // canvas interval in FP64
    double t0 = 0.0, t1 = __longlong_as_double(0x7FF0000000000000ll);
    bool miss = false;
    for (int a = 0; a < 3; ++a) {
        if (d64[a] != 0.0) {
            const double ta = (-T.half - o[a]) / d64[a], tb = (T.half - o[a]) / d64[a];
            t0 = fmax(t0, d64[a] > 0.0 ? ta : tb);
            t1 = fmin(t1, d64[a] > 0.0 ? tb : ta);
        } else if (!(o[a] >= -T.half && o[a] < T.half)) {
            miss = true;
        }
    }
    float C[3] = {0.f, 0.f, 0.f}, Tr = 1.f;
    int steps = 0;
    unsigned long long leaf_loads = 0, rec_loads = 0;
    double angle = 0.0;
    if (!miss && t0 < t1) {
        // start leaf at t0+ (FP64 point location, as in the other kernels)
        unsigned c[3] = {0u, 0u, 0u};
        int L = 0;
        int32_t rec = 0, slot;
        int32_t srec = 0;  // record and child index of the current leaf's slot
        int sk = 0;
        for (;;) {
            const double w = T.extent * p2d(-(L + 1));
            int k = 0;
            for (int a = 0; a < 3; ++a) {
                const double M = fma((double)(2u * c[a] + 1u), w, -T.half);
                unsigned b;
                if (d64[a] > 0.0) b = (M - o[a]) / d64[a] <= t0;
                else if (d64[a] < 0.0) b = (M - o[a]) / d64[a] > t0;
                else b = o[a] >= M;
                c[a] = 2u * c[a] + b;
                k |= (int)b << a;
            }
            slot = __ldg(T.nodes + (long long)rec * 8 + k);
            rec_loads += 1;
            ++L;
            srec = rec;
            sk = k;
            if (slot <= 0) break;
            rec = slot;
        }
        const GT d[3] = {G::from_d(d64[0]), G::from_d(d64[1]), G::from_d(d64[2])};
        const GT g_half = G::from_f(0.5f), g_mhalf = G::from_f(-0.5f), g_two = G::from_f(2.0f);
        GT p[3];
        for (int a = 0; a < 3; ++a) {
            const double x = fma(t0, d64[a], o[a]);
            if (kCellLocal) {
                const double w = T.extent * p2d(-L);
                const double centre = fma((double)c[a] + 0.5, w, -T.half);
                p[a] = G::from_d((x - centre) / w);  // start point in the cell frame: the error e0
            } else {
                p[a] = G::from_d(x);                 // start point snapped to FP32 canvas coordinates
            }
        }
        double X[3] = {fma(t0, d64[0], o[0]), fma(t0, d64[1], o[1]), fma(t0, d64[2], o[2])};
        for (;;) {
            if (steps >= P.step_limit) {
                atomicOr(&P.scratch->status, 1ull);
                atomicAdd(&P.scratch->stats[kStatStepLimited], 1ull);
                break;
            }
            steps += 1;
            const double w64 = T.extent * p2d(-L);
            const float w = (float)w64;
            // exit face: t_a = (face_a - p_a) / d_a, the nearest one
            GT te = G::from_f(0.0f);
            float tef = __int_as_float(0x7F800000);
            int ax = -1;
            for (int a = 0; a < 3; ++a) {
                if (G::f(d[a]) == 0.0f) continue;
                GT face;
                if (kCellLocal) face = G::f(d[a]) > 0.0f ? g_half : g_mhalf;
                else face = G::from_d(fma((double)(c[a] + (G::f(d[a]) > 0.0f ? 1u : 0u)), w64, -T.half));
                const GT ta = G::div(G::sub(face, p[a]), d[a]);
                if (G::f(ta) < tef) { te = ta; tef = G::f(ta); ax = a; }
            }
            if (ax < 0) break;
            const float ell = kCellLocal ? __fmul_rn(fmaxf(tef, 0.0f), w) : fmaxf(tef, 0.0f);
            if (slot < 0) {
                const uint2 q = __ldg(T.leaves + leaf_index(T, srec, sk, slot));
                leaf_loads += 1;
                const float s = h2f32((unsigned short)(q.y >> 16));
                if (s > 0.0f) {
                    const float a = -expm1f(-s * ell);
                    C[0] += Tr * a * h2f32((unsigned short)(q.x & 0xFFFFu));
                    C[1] += Tr * a * h2f32((unsigned short)(q.x >> 16));
                    C[2] += Tr * a * h2f32((unsigned short)(q.y & 0xFFFFu));
                    Tr *= expf(-s * ell);
                }
            }
            // exit point p' = p + t d (the exit axis on its face)
            GT pe[3];
            for (int a = 0; a < 3; ++a) pe[a] = G::add(p[a], G::mul(te, d[a]));
            if (kCellLocal) pe[ax] = G::f(d[ax]) > 0.0f ? g_half : g_mhalf;
            // final position so far, in FP64 canvas coordinates
            for (int a = 0; a < 3; ++a)
                X[a] = kCellLocal ? fma((double)c[a] + 0.5 + (double)G::f(pe[a]), w64, -T.half) : (double)G::f(pe[a]);
            if (Tr < P.t_min) break;
            const unsigned up = G::f(d[ax]) > 0.0f ? 1u : 0u;
            const unsigned cn = up ? c[ax] + 1u : c[ax] - 1u;
            if ((cn >> L) != 0u) break;  // leaves the canvas
            unsigned cc[3] = {c[0], c[1], c[2]};
            cc[ax] = cn;
            int Ln, kk;
            int32_t pr;
            slot = locate_int(T, cc, L, &Ln, &pr, &kk, &rec_loads);
            srec = pr;
            sk = kk;
            // position in the frame of the same-level neighbour (its centre is one cell further on ax)
            GT q[3];
            for (int a = 0; a < 3; ++a) q[a] = pe[a];
            if (kCellLocal) q[ax] = up ? g_mhalf : g_half;
            int Lc = L;
            while (slot > 0) {
                // finer neighbour: near side on the exit axis, FP32 position on the others
                rec = slot;
                int k = 0;
                const double wc = T.extent * p2d(-(Lc + 1));
                for (int a = 0; a < 3; ++a) {
                    unsigned b;
                    if (a == ax) {
                        b = up ? 0u : 1u;
                    } else if (kCellLocal) {
                        b = G::f(q[a]) > 0.0f || (G::f(q[a]) == 0.0f && G::f(d[a]) >= 0.0f);
                    } else {
                        const float M = G::f(G::from_d(fma((double)(2u * cc[a] + 1u), wc, -T.half)));
                        b = G::f(q[a]) > M || (G::f(q[a]) == M && G::f(d[a]) >= 0.0f);
                    }
                    if (kCellLocal) q[a] = G::sub(G::mul(g_two, q[a]), b ? g_half : g_mhalf);
                    cc[a] = 2u * cc[a] + b;
                    k |= (int)b << a;
                }
                ++Lc;
                slot = __ldg(T.nodes + (long long)rec * 8 + k);
                rec_loads += 1;
                srec = rec;
                sk = k;
                Ln = Lc;
            }
            if (kCellLocal && Ln < L) {
                // coarser neighbour: p s + c with s = 2^(Ln - L) and c the centre offset (exact)
                const double s64 = p2d(Ln - L);
                const GT s = G::from_d(s64);  // binary16: 0 below 2^-25 (the offset alone then places the point)
                for (int a = 0; a < 3; ++a) {
                    const unsigned cp = cc[a] >> (L - Ln);
                    const double off = ((double)cc[a] + 0.5) * s64 - ((double)cp + 0.5);
                    q[a] = G::add(G::mul(q[a], s), G::from_d(off));
                }
                if (kCellLocal) q[ax] = up ? g_mhalf : g_half;
            }
            const int sh = Lc - Ln;
            for (int a = 0; a < 3; ++a) {
                c[a] = cc[a] >> sh;
                p[a] = q[a];
            }
            L = Ln;
        }
        // angle between the initial direction and the eye-to-final-position line
        const double v[3] = {X[0] - o[0], X[1] - o[1], X[2] - o[2]};
        const double cx = v[1] * d64[2] - v[2] * d64[1], cy = v[2] * d64[0] - v[0] * d64[2], cz = v[0] * d64[1] - v[1] * d64[0];
        const double dt = v[0] * d64[0] + v[1] * d64[1] + v[2] * d64[2];
        angle = atan2(sqrt(cx * cx + cy * cy + cz * cz), dt) * 57.29577951308232;
    }
    float4 out;
    out.x = C[0] + Tr * V.bg[0];
    out.y = C[1] + Tr * V.bg[1];
    out.z = C[2] + Tr * V.bg[2];
    out.w = 1.0f - Tr;
    const long long pix = V.out_offset + idx;
    P.out[pix] = out;
    if (P.step_count) P.step_count[pix] = steps;
    if (P.angle_deg) P.angle_deg[pix] = (float)angle;
    return Local32Count{(unsigned long long)steps, leaf_loads, rec_loads};
}

template <bool kCellLocal, typename G>
__global__ void __launch_bounds__(256) local32_kernel(PlainParams P, long long n_pixels) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    Local32Count c = {0ull, 0ull, 0ull};
    const bool valid = idx < n_pixels;
    if (valid) c = local32_ray<kCellLocal, G>(P, idx);
    unsigned long long vals[5] = {valid ? 1ull : 0ull, c.steps, 0ull, c.leaf_loads, c.rec_loads};
    for (int q = 0; q < 5; ++q) {
        unsigned long long s = vals[q];
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, off);
        if ((threadIdx.x & 31) == 0 && s) atomicAdd(&P.scratch->stats[q], s);
    }
}

}  // namespace

cudaError_t launch_local32(const PlainParams& p, int precision, long long n_pixels, cudaStream_t s) {
    if (n_pixels <= 0) return cudaSuccess;
    const long long grid = (n_pixels + 255) / 256;
    if (grid > 0x7FFFFFFFll) return cudaErrorInvalidValue;
    if (precision == CANVOX_PREC_CELL32) local32_kernel<true, Geo32><<<(unsigned)grid, 256, 0, s>>>(p, n_pixels);
    else if (precision == CANVOX_PREC_CELL16) local32_kernel<true, Geo16><<<(unsigned)grid, 256, 0, s>>>(p, n_pixels);
    else local32_kernel<false, Geo32><<<(unsigned)grid, 256, 0, s>>>(p, n_pixels);
    return cudaGetLastError();
}

}  // namespace canvox
