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
// Both write, per pixel and on request, the angle between the initial ray
// direction and the line from the eye to the ray's final position (degrees).
// The eye and the pixel ray are the FP64 camera model; the start leaf is
// located in FP64 as in the other kernels; leaves are located from the root
// each step from integer coordinates, and by the FP32 position below the
// level of the cell the ray leaves.
#include "canvox_internal.cuh"

namespace canvox {
namespace {

__device__ __forceinline__ float h2f32(unsigned short h) {
    const float m = __int_as_float((int)((h & 0x7FFFu) << 13)) * 5.192296858534828e+33f;  // * 2^112
    return __int_as_float(__float_as_int(m) | (int)((h & 0x8000u) << 16));
}
__device__ __forceinline__ double p2d(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }

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

template <bool kCellLocal>
__device__ Local32Count local32_ray(const PlainParams& P, long long idx) {
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
            if (slot <= 0) break;
            rec = slot;
        }
        const float d[3] = {(float)d64[0], (float)d64[1], (float)d64[2]};
        float p[3];
        for (int a = 0; a < 3; ++a) {
            const double x = fma(t0, d64[a], o[a]);
            if (kCellLocal) {
                const double w = T.extent * p2d(-L);
                const double centre = fma((double)c[a] + 0.5, w, -T.half);
                p[a] = (float)((x - centre) / w);  // start point in the cell frame: the error e0
            } else {
                p[a] = (float)x;                   // start point snapped to FP32 canvas coordinates
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
            float te = __int_as_float(0x7F800000);
            int ax = -1;
            for (int a = 0; a < 3; ++a) {
                if (d[a] == 0.0f) continue;
                float face;
                if (kCellLocal) face = d[a] > 0.0f ? 0.5f : -0.5f;
                else face = (float)fma((double)(c[a] + (d[a] > 0.0f ? 1u : 0u)), w64, -T.half);
                const float ta = __fdiv_rn(__fsub_rn(face, p[a]), d[a]);
                if (ta < te) { te = ta; ax = a; }
            }
            if (ax < 0) break;
            const float ell = kCellLocal ? __fmul_rn(fmaxf(te, 0.0f), w) : fmaxf(te, 0.0f);
            if (slot < 0) {
                const uint2 q = __ldg(T.leaves + (-(long long)slot - 1));
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
            float pe[3];
            for (int a = 0; a < 3; ++a) pe[a] = __fadd_rn(p[a], __fmul_rn(te, d[a]));
            if (kCellLocal) pe[ax] = d[ax] > 0.0f ? 0.5f : -0.5f;
            // final position so far, in FP64 canvas coordinates
            for (int a = 0; a < 3; ++a)
                X[a] = kCellLocal ? fma((double)c[a] + 0.5 + (double)pe[a], w64, -T.half) : (double)pe[a];
            if (Tr < P.t_min) break;
            const unsigned up = d[ax] > 0.0f ? 1u : 0u;
            const unsigned cn = up ? c[ax] + 1u : c[ax] - 1u;
            if ((cn >> L) != 0u) break;  // leaves the canvas
            unsigned cc[3] = {c[0], c[1], c[2]};
            cc[ax] = cn;
            int Ln, kk;
            int32_t pr;
            slot = locate_int(T, cc, L, &Ln, &pr, &kk, &rec_loads);
            // position in the frame of the same-level neighbour (its centre is one cell further on ax)
            float q[3];
            for (int a = 0; a < 3; ++a) q[a] = pe[a];
            if (kCellLocal) q[ax] = up ? -0.5f : 0.5f;
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
                        b = q[a] > 0.0f || (q[a] == 0.0f && d[a] >= 0.0f);
                    } else {
                        const float M = (float)fma((double)(2u * cc[a] + 1u), wc, -T.half);
                        b = q[a] > M || (q[a] == M && d[a] >= 0.0f);
                    }
                    if (kCellLocal) q[a] = __fsub_rn(__fmul_rn(2.0f, q[a]), b ? 0.5f : -0.5f);
                    cc[a] = 2u * cc[a] + b;
                    k |= (int)b << a;
                }
                ++Lc;
                slot = __ldg(T.nodes + (long long)rec * 8 + k);
                rec_loads += 1;
                Ln = Lc;
            }
            if (kCellLocal && Ln < L) {
                // coarser neighbour: p s + c with s = 2^(Ln - L) and c the centre offset (exact)
                const float s = __int_as_float((127 + (Ln - L)) << 23);
                for (int a = 0; a < 3; ++a) {
                    const unsigned cp = cc[a] >> (L - Ln);
                    const double off = ((double)cc[a] + 0.5) * (double)s - ((double)cp + 0.5);
                    q[a] = __fadd_rn(__fmul_rn(q[a], s), (float)off);
                }
                if (kCellLocal) q[ax] = up ? -0.5f : 0.5f;
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

template <bool kCellLocal>
__global__ void __launch_bounds__(256) local32_kernel(PlainParams P, long long n_pixels) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    Local32Count c = {0ull, 0ull, 0ull};
    const bool valid = idx < n_pixels;
    if (valid) c = local32_ray<kCellLocal>(P, idx);
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
    if (precision == CANVOX_PREC_CELL32) local32_kernel<true><<<(unsigned)grid, 256, 0, s>>>(p, n_pixels);
    else local32_kernel<false><<<(unsigned)grid, 256, 0, s>>>(p, n_pixels);
    return cudaGetLastError();
}

}  // namespace canvox
