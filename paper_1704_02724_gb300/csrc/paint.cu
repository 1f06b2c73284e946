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
// descend (undecided) or already paint its whole subtree (painted); one warp
// per refined cell classifies that list against its eight children, 32
// entries at a time (a cell around a room holds tens of thousands of stamps),
// with each stamp's distances to the cell's three planes per axis shared by
// the children. Levels of few cells take a warp per child instead, and cells
// whose lists run long (near the root every stamp is on them; around a room,
// its stamps) a warp per chunk of a child's list. Geometry is FP64 with the
// same operations and order as the host painter, so the pools are identical.
#include <algorithm>
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

enum { kDrop = 0, kPaint = 1, kKeep = 2 };

// Lanes take a cell's stamp list 32 entries at a time, in order.
constexpr unsigned kFullMask = 0xFFFFFFFFu;
constexpr int kWarpsPerBlock = 4;
constexpr int64_t kSplitCells = 8192;  // levels with fewer refined cells take one warp per child

// One warp per refined cell, all eight children at once. Per axis a stamp's squared distances to the
// cell's three planes (low, mid, high) serve both halves, so a child's box distances are sums of
// per-axis terms already formed: (t0 + t1) + t2, the host painter's sums with its zero terms dropped,
// which leaves them bit-identical (adding +0 is exact).
struct ParentTerms {
    double dmin[2][3], dmax[2][3];  // [bit][axis]
    double cen[2][3];               // squared distance to the child centre's coordinate
};

__device__ __forceinline__ void parent_terms(const double* c, const double pl[3], const double pm[3], const double pu[3],
                                             const double cl[3], const double cm[3], ParentTerms& T) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double A = sq(__dsub_rn(c[a], pl[a])), B = sq(__dsub_rn(c[a], pm[a])), C = sq(__dsub_rn(c[a], pu[a]));
        T.dmin[0][a] = c[a] < pl[a] ? A : (c[a] > pm[a] ? B : 0.0);
        T.dmin[1][a] = c[a] < pm[a] ? B : (c[a] > pu[a] ? C : 0.0);
        T.dmax[0][a] = fmax(A, B);
        T.dmax[1][a] = fmax(B, C);
        T.cen[0][a] = sq(__dsub_rn(cl[a], c[a]));
        T.cen[1][a] = sq(__dsub_rn(cm[a], c[a]));
    }
}

// Term of child k on axis a (the half it lies in), picked without indexing by a runtime value.
template <typename V>
__device__ __forceinline__ V half_term(const V (&x)[2][3], int k, int a) {
    return ((k >> a) & 1) ? x[1][a] : x[0][a];
}

// Child k: kDrop / kPaint / kKeep for an undecided stamp with squared radius r2.
__device__ __forceinline__ int classify_child(const ParentTerms& T, int k, double r2, bool refined) {
    const double dmin2 = __dadd_rn(__dadd_rn(half_term(T.dmin, k, 0), half_term(T.dmin, k, 1)), half_term(T.dmin, k, 2));
    if (dmin2 >= r2) return kDrop;
    const double dmax2 = __dadd_rn(__dadd_rn(half_term(T.dmax, k, 0), half_term(T.dmax, k, 1)), half_term(T.dmax, k, 2));
    if (dmax2 <= r2) return kPaint;
    if (refined) return kKeep;
    const double d2 = __dadd_rn(__dadd_rn(half_term(T.cen, k, 0), half_term(T.cen, k, 1)), half_term(T.cen, k, 2));
    return d2 < r2 ? kPaint : kDrop;
}

// FP32 screen of the same box distances. Each coordinate difference to the low plane is formed in FP64 and
// rounded once; the rest is FP32. Every FP32 distance is within `margin` of its FP64 counterpart (a generous
// bound: differences within 2^-23 M_a, squares within 2^-21 M_a^2, two additions), so a comparison with r2
// farther than `margin` decides as the FP64 one does; closer ones are retaken in FP64.
struct FastTerms {
    float dmin[2][3], dmax[2][3], cen[2][3];
    float r2, margin;
};

__device__ __forceinline__ void fast_terms(const double* c, const double pl[3], float h, float hh, double r2,
                                           FastTerms& F) {
    float mm = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float dl = __double2float_rn(__dsub_rn(c[a], pl[a]));
        const float dm = __fsub_rn(dl, h), du = __fsub_rn(dm, h);
        const float A = __fmul_rn(dl, dl), B = __fmul_rn(dm, dm), C = __fmul_rn(du, du);
        F.dmin[0][a] = dl < 0.0f ? A : (dm > 0.0f ? B : 0.0f);
        F.dmin[1][a] = dm < 0.0f ? B : (du > 0.0f ? C : 0.0f);
        F.dmax[0][a] = fmaxf(A, B);
        F.dmax[1][a] = fmaxf(B, C);
        const float el = __fsub_rn(dl, hh), em = __fsub_rn(dm, hh);
        F.cen[0][a] = __fmul_rn(el, el);
        F.cen[1][a] = __fmul_rn(em, em);
        const float M = fabsf(dl) + 2.0f * h;
        mm = __fmaf_rn(M, M, mm);
    }
    F.r2 = __double2float_rn(r2);
    F.margin = 3.814697265625e-06f * mm + 2.384185791015625e-07f * F.r2;  // 2^-18 sum M^2 + 2^-22 r2
}

// kDrop / kPaint / kKeep when the screen decides, -1 when FP64 must.
__device__ __forceinline__ int classify_fast(const FastTerms& F, int k, bool refined) {
    const float lo = F.r2 - F.margin, hi = F.r2 + F.margin;
    const float dmin2 = (half_term(F.dmin, k, 0) + half_term(F.dmin, k, 1)) + half_term(F.dmin, k, 2);
    if (dmin2 >= hi) return kDrop;
    if (dmin2 >= lo) return -1;
    const float dmax2 = (half_term(F.dmax, k, 0) + half_term(F.dmax, k, 1)) + half_term(F.dmax, k, 2);
    if (dmax2 <= lo) return kPaint;
    if (dmax2 <= hi) return -1;
    if (refined) return kKeep;
    const float d2 = (half_term(F.cen, k, 0) + half_term(F.cen, k, 1)) + half_term(F.cen, k, 2);
    if (d2 < lo) return kPaint;
    if (d2 >= hi) return kDrop;
    return -1;
}

// Partial cover (the refining test): 1 / 0 when the screen decides, -1 when FP64 must.
__device__ __forceinline__ int partial_fast(const FastTerms& F, int k) {
    const float lo = F.r2 - F.margin, hi = F.r2 + F.margin;
    const float dmin2 = (half_term(F.dmin, k, 0) + half_term(F.dmin, k, 1)) + half_term(F.dmin, k, 2);
    if (dmin2 >= hi) return 0;
    if (dmin2 >= lo) return -1;
    const float dmax2 = (half_term(F.dmax, k, 0) + half_term(F.dmax, k, 1)) + half_term(F.dmax, k, 2);
    if (dmax2 <= lo) return 0;
    if (dmax2 <= hi) return -1;
    return 1;
}

__device__ __forceinline__ void parent_planes(const LevelIn& L, int64_t i, double extent, double half, double pl[3],
                                              double pm[3], double pu[3], double cl[3], double cm[3]) {
    const double H = extent * __longlong_as_double((long long)(1023 - L.level) << 52);
    const double h = 0.5 * H, hh = 0.5 * h;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        pl[a] = fma((double)L.coord[3 * i + a], H, -half);  // exact: multiples of the cell size
        pm[a] = __dadd_rn(pl[a], h);
        pu[a] = __dadd_rn(pm[a], h);
        cl[a] = __dadd_rn(pl[a], hh);
        cm[a] = __dadd_rn(pm[a], hh);
    }
}

__global__ void __launch_bounds__(32 * kWarpsPerBlock) expand_parent_count(LevelIn L, StampDev S, int32_t depth,
                                                                           double extent, double half, int32_t* firstref,
                                                                           uint64_t* slot, int64_t* count, int64_t* is_int,
                                                                           const uint8_t* skip) {
    __shared__ int32_t s_idx[kWarpsPerBlock][32];
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (i >= L.n || (skip && skip[i])) return;  // warp-uniform (skipped cells take the chunked passes)
    double pl[3], pm[3], pu[3], cl[3], cm[3];
    parent_planes(L, i, extent, half, pl, pm, pu, cl, cm);
    const float hf = (float)(pm[0] - pl[0]), hhf = 0.5f * hf;  // child side and half side (exact)
    const int lc = L.level + 1;
    const int64_t b = L.off[i], e = L.off[i + 1];
    // the first refining stamp of each child
    int32_t fr[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) fr[k] = 0x7FFFFFFF;
    unsigned found = 0;
    if (lc < depth) {
        for (int64_t base = b; base < e && found != 0xFFu; base += 32) {
            const int64_t q = base + lane;
            int32_t v = -1;
            bool cand = false;
            FastTerms F;
            double r2 = 0.0;
            if (q < e) {
                v = L.ent[q];
                if (v >= 0 && S.kt[v] > lc) {
                    cand = true;
                    r2 = S.r2[v];
                    fast_terms(S.c + 3 * (int64_t)v, pl, hf, hhf, r2, F);
                }
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                bool qual = false;
                if (cand) {
                    const int f = partial_fast(F, k);
                    if (f >= 0) {
                        qual = f == 1;
                    } else {
                        ParentTerms T;
                        parent_terms(S.c + 3 * (int64_t)v, pl, pm, pu, cl, cm, T);
                        const double dmin2 = __dadd_rn(__dadd_rn(half_term(T.dmin, k, 0), half_term(T.dmin, k, 1)),
                                                       half_term(T.dmin, k, 2));
                        const double dmax2 = __dadd_rn(__dadd_rn(half_term(T.dmax, k, 0), half_term(T.dmax, k, 1)),
                                                       half_term(T.dmax, k, 2));
                        qual = dmin2 < r2 && dmax2 > r2;
                    }
                }
                const unsigned m = __ballot_sync(kFullMask, qual);
                const int32_t first = __shfl_sync(kFullMask, v, m ? __ffs(m) - 1 : 0);
                if (m && !((found >> k) & 1u)) {
                    fr[k] = first;
                    found |= 1u << k;
                }
            }
        }
    }
    // counts of the refined children, blends of the leaf children (lane k folds child k)
    int64_t n[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) n[k] = 0;
    float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t base = b; base < e; base += 32) {
        const int64_t q = base + lane;
        int32_t v = 0;
        bool valid = false;
        FastTerms F;
        double r2 = 0.0;
        if (q < e) {
            valid = true;
            v = L.ent[q];
            if (v >= 0) {
                r2 = S.r2[v];
                fast_terms(S.c + 3 * (int64_t)v, pl, hf, hhf, r2, F);
            }
        }
        s_idx[wib][lane] = v < 0 ? ~v : v;
        unsigned pmask = 0;  // lane k: the entries that paint leaf child k
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const bool internal = fr[k] != 0x7FFFFFFF;
            int c = kDrop;
            if (valid) {
                if (v < 0) {
                    c = kPaint;
                } else {
                    const bool refined = internal && fr[k] <= v;
                    c = classify_fast(F, k, refined);
                    if (c < 0) {
                        ParentTerms T;
                        parent_terms(S.c + 3 * (int64_t)v, pl, pm, pu, cl, cm, T);
                        c = classify_child(T, k, r2, refined);
                    }
                }
            }
            if (internal) {
                n[k] += __popc(__ballot_sync(kFullMask, c != kDrop));
            } else {
                const unsigned m = __ballot_sync(kFullMask, c == kPaint);
                if (lane == k) pmask = m;
            }
        }
        __syncwarp();
        if (lane < 8) {
            while (pmask) {
                const int j = __ffs(pmask) - 1;
                pmask &= pmask - 1;
                blend(val, S.rgba[s_idx[wib][j]]);
            }
        }
        __syncwarp();
    }
    if (lane < 8) {
        int64_t nk = 0;
        int32_t fk = 0x7FFFFFFF;
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (lane == k) {
                nk = n[k];
                fk = fr[k];
            }
        const int64_t t = 8 * i + lane;
        firstref[t] = fk;
        if (fk != 0x7FFFFFFF) {
            count[t] = nk;
            is_int[t] = 1;
            slot[t] = kInternal;
        } else {
            count[t] = 0;
            is_int[t] = 0;
            slot[t] = leaf_key(val);
        }
    }
}

__global__ void __launch_bounds__(32 * kWarpsPerBlock) expand_parent_write(LevelIn L, StampDev S, double extent,
                                                                           double half, const int32_t* firstref,
                                                                           uint64_t* slot, const int64_t* ent_off,
                                                                           const int64_t* next_idx, uint32_t* ncoord,
                                                                           int64_t* noff, int32_t* nent, const uint8_t* skip) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= L.n || (skip && skip[i])) return;
    int32_t fr[8];
    int64_t w[8];
    unsigned internal = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        fr[k] = firstref[8 * i + k];
        w[k] = ent_off[8 * i + k];
        if (slot[8 * i + k] == kInternal) internal |= 1u << k;
    }
    if (!internal) return;  // warp-uniform
    __syncwarp();
    if (lane < 8 && ((internal >> lane) & 1u)) {
        const int64_t t = 8 * i + lane, j = next_idx[t];
        slot[t] = kInternal | (uint64_t)j;
        ncoord[3 * j] = 2u * L.coord[3 * i] + (lane & 1u);
        ncoord[3 * j + 1] = 2u * L.coord[3 * i + 1] + ((lane >> 1) & 1u);
        ncoord[3 * j + 2] = 2u * L.coord[3 * i + 2] + ((lane >> 2) & 1u);
        noff[j] = ent_off[t];
    }
    double pl[3], pm[3], pu[3], cl[3], cm[3];
    parent_planes(L, i, extent, half, pl, pm, pu, cl, cm);
    const float hf = (float)(pm[0] - pl[0]), hhf = 0.5f * hf;
    const int64_t b = L.off[i], e = L.off[i + 1];
    for (int64_t base = b; base < e; base += 32) {
        const int64_t q = base + lane;
        int32_t v = 0;
        bool valid = false;
        FastTerms F;
        double r2 = 0.0;
        if (q < e) {
            valid = true;
            v = L.ent[q];
            if (v >= 0) {
                r2 = S.r2[v];
                fast_terms(S.c + 3 * (int64_t)v, pl, hf, hhf, r2, F);
            }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (!((internal >> k) & 1u)) continue;  // warp-uniform
            int c = kDrop;
            if (valid) {
                if (v < 0) {
                    c = kPaint;
                } else {
                    c = classify_fast(F, k, fr[k] <= v);
                    if (c < 0) {
                        ParentTerms T;
                        parent_terms(S.c + 3 * (int64_t)v, pl, pm, pu, cl, cm, T);
                        c = classify_child(T, k, r2, fr[k] <= v);
                    }
                }
            }
            const bool keep = c != kDrop;
            const unsigned m = __ballot_sync(kFullMask, keep);
            if (keep) nent[w[k] + __popc(m & ((1u << lane) - 1u))] = (v < 0 || c == kKeep) ? v : ~v;
            w[k] += __popc(m);
        }
    }
}

// Squared radius and target depth of each stamp: the smallest k with extent 2^-k <= r/10, at most depth.
__global__ void stamp_prep(const double* r, int64_t n, int32_t depth, double extent, double* r2, int32_t* kt) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const double rs = r[s];
    r2[s] = __dmul_rn(rs, rs);
    const double tgt = __ddiv_rn(rs, 10.0);
    int32_t k = 0;
    double w = extent;
    while (k < depth && w > tgt) {
        w = __dmul_rn(w, 0.5);
        ++k;
    }
    kt[s] = k;
}

// The same two passes with one warp per child, for levels of few refined cells: near the root and around the
// rooms a cell's list holds tens of thousands of stamps, and eight warps per cell instead of one keep the GPU
// busy. The per-child decisions are the ones above (the same screen and FP64 fallback), so the output is too.
__device__ __forceinline__ int child_class(const StampDev& S, const FastTerms& F, int32_t v, double r2, int k,
                                           bool refined, const double pl[3], const double pm[3], const double pu[3],
                                           const double cl[3], const double cm[3]) {
    int c = classify_fast(F, k, refined);
    if (c < 0) {
        ParentTerms T;
        parent_terms(S.c + 3 * (int64_t)v, pl, pm, pu, cl, cm, T);
        c = classify_child(T, k, r2, refined);
    }
    return c;
}

__global__ void __launch_bounds__(32 * kWarpsPerBlock) expand_child_count(LevelIn L, StampDev S, int32_t depth,
                                                                          double extent, double half, int32_t* firstref,
                                                                          uint64_t* slot, int64_t* count, int64_t* is_int,
                                                                          const uint8_t* skip) {
    __shared__ int32_t s_idx[kWarpsPerBlock][32];
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (t >= 8 * L.n || (skip && skip[t >> 3])) return;  // warp-uniform
    const int64_t i = t >> 3;
    const int k = (int)(t & 7);
    double pl[3], pm[3], pu[3], cl[3], cm[3];
    parent_planes(L, i, extent, half, pl, pm, pu, cl, cm);
    const float hf = (float)(pm[0] - pl[0]), hhf = 0.5f * hf;
    const int lc = L.level + 1;
    const int64_t b = L.off[i], e = L.off[i + 1];
    int32_t fr = 0x7FFFFFFF;
    if (lc < depth) {
        for (int64_t base = b; base < e; base += 32) {
            const int64_t q = base + lane;
            int32_t v = -1;
            bool qual = false;
            if (q < e) {
                v = L.ent[q];
                if (v >= 0 && S.kt[v] > lc) {
                    const double r2 = S.r2[v];
                    FastTerms F;
                    fast_terms(S.c + 3 * (int64_t)v, pl, hf, hhf, r2, F);
                    const int f = partial_fast(F, k);
                    if (f >= 0) {
                        qual = f == 1;
                    } else {
                        ParentTerms T;
                        parent_terms(S.c + 3 * (int64_t)v, pl, pm, pu, cl, cm, T);
                        const double dmin2 = __dadd_rn(__dadd_rn(half_term(T.dmin, k, 0), half_term(T.dmin, k, 1)),
                                                       half_term(T.dmin, k, 2));
                        const double dmax2 = __dadd_rn(__dadd_rn(half_term(T.dmax, k, 0), half_term(T.dmax, k, 1)),
                                                       half_term(T.dmax, k, 2));
                        qual = dmin2 < r2 && dmax2 > r2;
                    }
                }
            }
            const unsigned m = __ballot_sync(kFullMask, qual);
            if (m) {
                fr = __shfl_sync(kFullMask, v, __ffs(m) - 1);  // entries are in stamp order
                break;
            }
        }
    }
    int64_t n = 0;
    float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t base = b; base < e; base += 32) {
        const int64_t q = base + lane;
        int32_t v = 0;
        int c = kDrop;
        if (q < e) {
            v = L.ent[q];
            if (v < 0) {
                c = kPaint;
            } else {
                const double r2 = S.r2[v];
                FastTerms F;
                fast_terms(S.c + 3 * (int64_t)v, pl, hf, hhf, r2, F);
                c = child_class(S, F, v, r2, k, fr != 0x7FFFFFFF && fr <= v, pl, pm, pu, cl, cm);
            }
        }
        if (fr != 0x7FFFFFFF) {
            n += __popc(__ballot_sync(kFullMask, c != kDrop));
        } else {
            s_idx[wib][lane] = v < 0 ? ~v : v;
            unsigned m = __ballot_sync(kFullMask, c == kPaint);
            __syncwarp();
            while (m) {  // every lane folds the same sequence
                const int j = __ffs(m) - 1;
                m &= m - 1;
                blend(val, S.rgba[s_idx[wib][j]]);
            }
            __syncwarp();
        }
    }
    if (lane == 0) {
        firstref[t] = fr;
        if (fr != 0x7FFFFFFF) {
            count[t] = n;
            is_int[t] = 1;
            slot[t] = kInternal;
        } else {
            count[t] = 0;
            is_int[t] = 0;
            slot[t] = leaf_key(val);
        }
    }
}

__global__ void __launch_bounds__(32 * kWarpsPerBlock) expand_child_write(LevelIn L, StampDev S, double extent,
                                                                          double half, const int32_t* firstref,
                                                                          uint64_t* slot, const int64_t* ent_off,
                                                                          const int64_t* next_idx, uint32_t* ncoord,
                                                                          int64_t* noff, int32_t* nent, const uint8_t* skip) {
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= 8 * L.n || (skip && skip[t >> 3])) return;
    if (slot[t] != kInternal) return;  // warp-uniform
    const int64_t i = t >> 3;
    const int k = (int)(t & 7);
    const int32_t fr = firstref[t];
    const int64_t j = next_idx[t];
    int64_t w = ent_off[t];
    __syncwarp();
    if (lane == 0) {
        slot[t] = kInternal | (uint64_t)j;
        ncoord[3 * j] = 2u * L.coord[3 * i] + (k & 1u);
        ncoord[3 * j + 1] = 2u * L.coord[3 * i + 1] + ((k >> 1) & 1u);
        ncoord[3 * j + 2] = 2u * L.coord[3 * i + 2] + ((k >> 2) & 1u);
        noff[j] = w;
    }
    double pl[3], pm[3], pu[3], cl[3], cm[3];
    parent_planes(L, i, extent, half, pl, pm, pu, cl, cm);
    const float hf = (float)(pm[0] - pl[0]), hhf = 0.5f * hf;
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
                const double r2 = S.r2[v];
                FastTerms F;
                fast_terms(S.c + 3 * (int64_t)v, pl, hf, hhf, r2, F);
                const int c = child_class(S, F, v, r2, k, fr <= v, pl, pm, pu, cl, cm);
                keep = c != kDrop;
                out = c == kPaint ? ~v : v;
            }
        }
        const unsigned m = __ballot_sync(kFullMask, keep);
        if (keep) nent[w + __popc(m & ((1u << lane) - 1u))] = out;
        w += __popc(m);
    }
}

// The per-child passes once more, for the cells whose lists are long (near the root every stamp is on them, and
// around a room its tens of thousands of stamps are, level after level): a child's list is cut into chunks of
// kChunk entries, one warp each, so that such a cell runs on hundreds of warps instead of one (or eight). The
// first refining stamp is the least one any chunk finds (entries are in stamp order), the kept entries are counted
// per chunk and written at the child's list start plus the counts of its earlier chunks (which keeps every
// next-level list in stamp order), and a child that stays a leaf blends its painting stamps in order in one warp
// (such children of long lists rarely have any, and skip it). Every per-entry decision is the one of the passes
// above, so the pools are the same. The level's other cells take those passes, which skip the long ones.
constexpr int64_t kChunk = 2048;         // entries per warp
constexpr int64_t kChunkMinList = 8192;  // cells whose list is longer take the chunked passes
constexpr int32_t kNoStamp = 0x7FFFFFFF;

struct ChunkWork {
    int64_t t;      // child 8 i + k of refined cell i
    int64_t b, e;   // its entries [b, e) of cell i's list
    int64_t fw;     // index of the child's first chunk
    int32_t first;  // 1 for the child's first chunk
};

// Whether list entry v (a stamp that still descends) partially covers child k and has its target below level lc.
__device__ __forceinline__ bool refines_child(const StampDev& S, int32_t v, int k, int lc, const double pl[3],
                                              const double pm[3], const double pu[3], const double cl[3],
                                              const double cm[3], float hf, float hhf) {
    if (v < 0 || S.kt[v] <= lc) return false;
    const double r2 = S.r2[v];
    FastTerms F;
    fast_terms(S.c + 3 * (int64_t)v, pl, hf, hhf, r2, F);
    const int f = partial_fast(F, k);
    if (f >= 0) return f == 1;
    ParentTerms T;
    parent_terms(S.c + 3 * (int64_t)v, pl, pm, pu, cl, cm, T);
    const double dmin2 = __dadd_rn(__dadd_rn(half_term(T.dmin, k, 0), half_term(T.dmin, k, 1)), half_term(T.dmin, k, 2));
    const double dmax2 = __dadd_rn(__dadd_rn(half_term(T.dmax, k, 0), half_term(T.dmax, k, 1)), half_term(T.dmax, k, 2));
    return dmin2 < r2 && dmax2 > r2;
}

// kDrop / kPaint / kKeep of list entry x for child k whose first refining stamp is fr (kNoStamp: none).
__device__ __forceinline__ int entry_class(const StampDev& S, int32_t x, int k, int32_t fr, const double pl[3],
                                           const double pm[3], const double pu[3], const double cl[3],
                                           const double cm[3], float hf, float hhf) {
    if (x < 0) return kPaint;
    const double r2 = S.r2[x];
    FastTerms F;
    fast_terms(S.c + 3 * (int64_t)x, pl, hf, hhf, r2, F);
    return child_class(S, F, x, r2, k, fr != kNoStamp && fr <= x, pl, pm, pu, cl, cm);
}

// Cells with lists longer than kChunkMinList: skip[i] = flag[i] = 1.
__global__ void flag_long(LevelIn L, uint8_t* skip, int64_t* flag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L.n) return;
    const bool lg = L.off[i + 1] - L.off[i] > kChunkMinList;
    skip[i] = lg ? 1 : 0;
    flag[i] = lg ? 1 : 0;
}

// The long cells in order, as (cell, list start, list end); pos = exclusive scan of their flags.
__global__ void gather_long(LevelIn L, const uint8_t* skip, const int64_t* pos, int64_t* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L.n || !skip[i]) return;
    const int64_t j = pos[i];
    out[3 * j] = i;
    out[3 * j + 1] = L.off[i];
    out[3 * j + 2] = L.off[i + 1];
}

// Children of the long cells: cells[j >> 3] is the cell of the j-th.
__global__ void chunk_init(const int64_t* cells, int64_t nj, int32_t* fr, int64_t* cnt, int64_t* npaint) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nj) return;
    const int64_t t = 8 * cells[j >> 3] + (j & 7);
    fr[t] = kNoStamp;
    cnt[t] = 0;
    npaint[t] = 0;
}

__global__ void __launch_bounds__(32 * kWarpsPerBlock) chunk_firstref(LevelIn L, StampDev S, int32_t depth, double extent,
                                                                      double half, const ChunkWork* W, int64_t nw,
                                                                      int32_t* fr) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int lc = L.level + 1;
    if (w >= nw || lc >= depth) return;  // warp-uniform
    const ChunkWork cw = W[w];
    const int k = (int)(cw.t & 7);
    double pl[3], pm[3], pu[3], cl[3], cm[3];
    parent_planes(L, cw.t >> 3, extent, half, pl, pm, pu, cl, cm);
    const float hf = (float)(pm[0] - pl[0]), hhf = 0.5f * hf;
    for (int64_t base = cw.b; base < cw.e; base += 32) {
        const int64_t q = base + lane;
        const int32_t v = q < cw.e ? L.ent[q] : -1;
        const unsigned m = __ballot_sync(kFullMask, refines_child(S, v, k, lc, pl, pm, pu, cl, cm, hf, hhf));
        if (m) {
            const int32_t first = __shfl_sync(kFullMask, v, __ffs(m) - 1);
            if (lane == 0) atomicMin(&fr[cw.t], first);
            break;
        }
    }
}

// Per chunk: the entries a refined child keeps (chunk_cnt, summed into cnt), or the ones that paint a child that
// stays a leaf (summed into npaint).
__global__ void __launch_bounds__(32 * kWarpsPerBlock) chunk_count(LevelIn L, StampDev S, double extent, double half,
                                                                   const ChunkWork* W, int64_t nw, const int32_t* fr,
                                                                   int64_t* chunk_cnt, int64_t* cnt, int64_t* npaint) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nw) return;
    const ChunkWork cw = W[w];
    const int k = (int)(cw.t & 7);
    const int32_t f = fr[cw.t];
    double pl[3], pm[3], pu[3], cl[3], cm[3];
    parent_planes(L, cw.t >> 3, extent, half, pl, pm, pu, cl, cm);
    const float hf = (float)(pm[0] - pl[0]), hhf = 0.5f * hf;
    int64_t n = 0;
    for (int64_t base = cw.b; base < cw.e; base += 32) {
        const int64_t q = base + lane;
        const int c = q < cw.e ? entry_class(S, L.ent[q], k, f, pl, pm, pu, cl, cm, hf, hhf) : kDrop;
        n += __popc(__ballot_sync(kFullMask, f != kNoStamp ? c != kDrop : c == kPaint));
    }
    if (lane == 0) {
        chunk_cnt[w] = f != kNoStamp ? n : 0;
        if (n)
            atomicAdd(reinterpret_cast<unsigned long long*>(f != kNoStamp ? &cnt[cw.t] : &npaint[cw.t]),
                      (unsigned long long)n);
    }
}

// Per child: an internal slot, or the leaf key of the blend, in stamp order, of the stamps that paint it.
__global__ void __launch_bounds__(32 * kWarpsPerBlock) chunk_child_finish(LevelIn L, StampDev S, double extent, double half,
                                                                          const int64_t* cells, int64_t nj,
                                                                          const int32_t* fr, const int64_t* npaint,
                                                                          uint64_t* slot, int64_t* cnt, int64_t* is_int) {
    __shared__ int32_t s_idx[kWarpsPerBlock][32];
    const int64_t jj = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (jj >= nj) return;  // warp-uniform
    const int64_t t = 8 * cells[jj >> 3] + (jj & 7);
    if (fr[t] != kNoStamp) {
        if (lane == 0) {
            is_int[t] = 1;
            slot[t] = kInternal;
        }
        return;
    }
    float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
    if (npaint[t] > 0) {
        const int64_t i = t >> 3;
        const int k = (int)(t & 7);
        double pl[3], pm[3], pu[3], cl[3], cm[3];
        parent_planes(L, i, extent, half, pl, pm, pu, cl, cm);
        const float hf = (float)(pm[0] - pl[0]), hhf = 0.5f * hf;
        const int64_t b = L.off[i], e = L.off[i + 1];
        for (int64_t base = b; base < e; base += 32) {
            const int64_t q = base + lane;
            int32_t x = 0;
            int c = kDrop;
            if (q < e) {
                x = L.ent[q];
                c = entry_class(S, x, k, kNoStamp, pl, pm, pu, cl, cm, hf, hhf);
            }
            s_idx[wib][lane] = x < 0 ? ~x : x;
            unsigned m = __ballot_sync(kFullMask, c == kPaint);
            __syncwarp();
            while (m) {  // every lane folds the same sequence
                const int j = __ffs(m) - 1;
                m &= m - 1;
                blend(val, S.rgba[s_idx[wib][j]]);
            }
            __syncwarp();
        }
    }
    if (lane == 0) {
        cnt[t] = 0;
        is_int[t] = 0;
        slot[t] = leaf_key(val);
    }
}

// Per chunk of a refined child: its kept entries at the child's list start plus the kept entries of its earlier
// chunks (chunk_scan, the exclusive scan of chunk_cnt over all chunks); the child's first chunk also writes its
// cell and list start.
__global__ void __launch_bounds__(32 * kWarpsPerBlock) chunk_write(LevelIn L, StampDev S, double extent, double half,
                                                                   const ChunkWork* W, int64_t nw, const int32_t* fr,
                                                                   uint64_t* slot, const int64_t* ent_off,
                                                                   const int64_t* next_idx, const int64_t* chunk_scan,
                                                                   uint32_t* ncoord, int64_t* noff, int32_t* nent) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nw) return;
    const ChunkWork cw = W[w];
    const int32_t f = fr[cw.t];
    if (f == kNoStamp) return;  // a leaf child
    const int64_t i = cw.t >> 3;
    const int k = (int)(cw.t & 7);
    if (cw.first && lane == 0) {
        const int64_t j = next_idx[cw.t];
        slot[cw.t] = kInternal | (uint64_t)j;
        ncoord[3 * j] = 2u * L.coord[3 * i] + (k & 1u);
        ncoord[3 * j + 1] = 2u * L.coord[3 * i + 1] + ((k >> 1) & 1u);
        ncoord[3 * j + 2] = 2u * L.coord[3 * i + 2] + ((k >> 2) & 1u);
        noff[j] = ent_off[cw.t];
    }
    double pl[3], pm[3], pu[3], cl[3], cm[3];
    parent_planes(L, i, extent, half, pl, pm, pu, cl, cm);
    const float hf = (float)(pm[0] - pl[0]), hhf = 0.5f * hf;
    int64_t pos = ent_off[cw.t] + (chunk_scan[w] - chunk_scan[cw.fw]);
    for (int64_t base = cw.b; base < cw.e; base += 32) {
        const int64_t q = base + lane;
        int32_t out = 0;
        bool keep = false;
        if (q < cw.e) {
            const int32_t x = L.ent[q];
            if (x < 0) {
                out = x;
                keep = true;
            } else {
                const int c = entry_class(S, x, k, f, pl, pm, pu, cl, cm, hf, hhf);
                keep = c != kDrop;
                out = c == kPaint ? ~x : x;
            }
        }
        const unsigned m = __ballot_sync(kFullMask, keep);
        if (keep) nent[pos + __popc(m & ((1u << lane) - 1u))] = out;
        pos += __popc(m);
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
// Leaf numbers (breadth-first slot order) are written modulo 2^31; the slot position 8 r + k of each leaf
// whose number is a nonzero multiple m 2^31 goes to wraps[m - 1].
__global__ void write_level(int64_t n, const uint64_t* slot, const uint64_t* ckey_next, const int64_t* rec_scan,
                            const int64_t* leaf_scan, const int64_t* surv, int64_t rec_base, int64_t next_rec_base,
                            int64_t leaf_base, const int64_t* next_rec_scan, int32_t* nodes, uint2* leaves,
                            int64_t* wraps) {
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
                const int64_t low = lf & 0x7FFFFFFFll;
                out = -(int32_t)low - 1;
                if (low == 0 && lf > 0) wraps[(lf >> 31) - 1] = 8 * r + k;
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

// ---------------------------------------------------------------------------
// Partitions for appends. The refined cells of one level P (the partition level)
// split the tree: breadth-first order keeps each one's subtree contiguous within
// every deeper level, in the order of the partitions. Stamps appended later do
// not change what any earlier stamp does (a cell's first refining stamp can only
// appear among the new ones), so a partition whose stamp list at level P is
// unchanged keeps its whole subtree, and only the others are painted again.
// ---------------------------------------------------------------------------

// pid_next[child index] = pid[parent] for every internal child (the partition a cell belongs to).
__global__ void pid_propagate(int64_t n, const uint64_t* slot, const int32_t* pid, int32_t* pid_next) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 8 * n) return;
    const uint64_t v = slot[t];
    if (v & kInternal) pid_next[v & ~kInternal] = pid[t >> 3];
}

// off[p] = first index of partition p in the (nondecreasing) partition ids of one level, p = 0 .. nseg.
__global__ void seg_offsets(int64_t n, const int32_t* pid, int64_t nseg, int64_t* off) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p > nseg) return;
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (pid[mid] < p) lo = mid + 1;
        else hi = mid;
    }
    off[p] = lo;
}

__global__ void iota32(int64_t n, int32_t* v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = (int32_t)i;
}

// Morton code of a level-P cell: its child indices k = x + 2y + 4z from the root down, 3 bits per level (the
// breadth-first order of the level).
__device__ __forceinline__ uint64_t morton(const uint32_t* c, int P) {
    uint64_t m = 0;
    for (int b = P - 1; b >= 0; --b)
        m = (m << 3) | (uint64_t)(((c[0] >> b) & 1u) | (((c[1] >> b) & 1u) << 1) | (((c[2] >> b) & 1u) << 2));
    return m;
}
__global__ void morton_codes(int64_t n, const uint32_t* coord, int P, uint64_t* code) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) code[i] = morton(coord + 3 * i, P);
}

// One warp per new partition: the old partition with the same cell and the same stamp list (entry for entry),
// else -1.
__global__ void match_partitions(int64_t n_new, const uint32_t* coord_new, const int64_t* off_new,
                                 const int32_t* ent_new, int64_t n_old, const uint64_t* code_old,
                                 const int64_t* off_old, const int32_t* ent_old, int P, int32_t* reuse) {
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= n_new) return;  // warp-uniform
    const uint64_t m = morton(coord_new + 3 * p, P);
    int64_t lo = 0, hi = n_old;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (code_old[mid] < m) lo = mid + 1;
        else hi = mid;
    }
    int32_t q = -1;
    if (lo < n_old && code_old[lo] == m) {
        const int64_t bn = off_new[p], en = off_new[p + 1], bo = off_old[lo], eo = off_old[lo + 1];
        bool same = en - bn == eo - bo;
        for (int64_t j = lane; same && j < en - bn; j += 32)
            if (ent_new[bn + j] != ent_old[bo + j]) same = false;
        same = __all_sync(kFullMask, same);
        if (same) q = (int32_t)lo;
    }
    if (lane == 0) reuse[p] = q;
}

// Cells `sel` of a level (their coordinates and stamp lists) gathered into a new level; dst_off = exclusive scan of
// the selected lists' lengths.
__global__ void gather_cells(int64_t m, const int32_t* sel, const uint32_t* coord, const int64_t* off,
                             const int32_t* ent, const int64_t* dst_off, uint32_t* ncoord, int64_t* noff, int32_t* nent) {
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= m) return;
    const int64_t i = sel[r], b = off[i], e = off[i + 1], d = dst_off[r];
    if (lane < 3) ncoord[3 * r + lane] = coord[3 * i + lane];
    if (lane == 0) noff[r] = d;
    for (int64_t j = lane; j < e - b; j += 32) nent[d + j] = ent[b + j];
}
__global__ void list_lengths(int64_t m, const int32_t* sel, const int64_t* off, int64_t* len) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < m) len[r] = off[sel[r] + 1] - off[sel[r]];
}

// Per new partition p, its cell count at one level: from the kept subtree (reuse[p] = q) or the repainted one
// (rep[p] = r).
__global__ void part_counts(int64_t n, const int32_t* reuse, const int32_t* rep, const int64_t* off_old,
                            const int64_t* off_rep, int64_t* cnt) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int32_t q = reuse[p];
    cnt[p] = q >= 0 ? (off_old ? off_old[q + 1] - off_old[q] : 0) : (off_rep ? off_rep[rep[p] + 1] - off_rep[rep[p]] : 0);
}

// The assembled level: each cell's eight slots copied from its source, internal children renumbered to the
// assembled next level (same partition, same position within it).
__global__ void assemble_level(int64_t n_dst, int64_t n_part, const int64_t* dst_off, const int64_t* dst_off_next,
                               const int32_t* reuse, const int32_t* rep, const uint64_t* slot_old,
                               const int64_t* off_old, const int64_t* off_old_next, const uint64_t* slot_rep,
                               const int64_t* off_rep, const int64_t* off_rep_next, uint64_t* slot_dst) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 8 * n_dst) return;
    const int64_t j = t >> 3;
    int64_t lo = 0, hi = n_part;  // the partition p with dst_off[p] <= j < dst_off[p + 1]
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (dst_off[mid] <= j) lo = mid;
        else hi = mid;
    }
    const int64_t p = lo, local = j - dst_off[p];
    const int32_t q = reuse[p];
    uint64_t v;
    int64_t src_next;
    if (q >= 0) {
        v = slot_old[8 * (off_old[q] + local) + (t & 7)];
        src_next = (v & kInternal) ? off_old_next[q] : 0;
    } else {
        const int32_t r = rep[p];
        v = slot_rep[8 * (off_rep[r] + local) + (t & 7)];
        src_next = (v & kInternal) ? off_rep_next[r] : 0;
    }
    if (v & kInternal) v = kInternal | (uint64_t)((int64_t)(v & ~kInternal) - src_next + dst_off_next[p]);
    slot_dst[t] = v;
}

}  // namespace

#define PCK(call)                                    \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return e_;            \
    } while (0)

namespace {

// Merge of identical siblings and the breadth-first pools of the painted levels (slots[l]: 8 child slots per
// refined cell of level l), with the positions where leaf numbers pass multiples of 2^31.
cudaError_t finish_pools(const std::vector<uint64_t*>& slots, const std::vector<int64_t>& ncell, int32_t** d_nodes_out,
                         uint2** d_leaves_out, int64_t* n_rec_out, int64_t* n_leaf_out,
                         std::vector<int64_t>* level_begin, int64_t* wrap_out, int32_t* n_wrap_out) {
    DevBuf buf;
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
    if (n_rec > 0x7FFFFFFFll || n_leaf > kMaxLeaves) return cudaErrorMemoryAllocation;  // beyond the pool format
    const int32_t n_wrap = n_leaf > 0 ? (int32_t)((n_leaf - 1) >> 31) : 0;
    int64_t* d_wraps;
    PCK(buf.alloc(&d_wraps, kMaxWraps));
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
                                                   l + 1 < nl ? rec_scan[(size_t)l + 1] : zero_scan, d_nodes, d_leaves,
                                                   d_wraps);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess && n_wrap > 0)
        e = cudaMemcpy(wrap_out, d_wraps, sizeof(int64_t) * (size_t)n_wrap, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        cudaFree(d_nodes);
        cudaFree(d_leaves);
        return e;
    }
    *n_wrap_out = n_wrap;
    *d_nodes_out = d_nodes;
    *d_leaves_out = d_leaves;
    *n_rec_out = n_rec;
    *n_leaf_out = n_leaf;
    level_begin->clear();
    for (int l = 0; l <= nl; ++l)
        if (l == 0 || rec_base[(size_t)l] > rec_base[(size_t)l - 1]) level_begin->push_back(rec_base[(size_t)l]);
    return cudaSuccess;
}

}  // namespace

namespace {

// Refined cells of one level with their ordered stamp lists (device arrays owned here).
struct Level {
    int64_t n = 0;
    int32_t level = 0;
    uint32_t* coord = nullptr;  // [n][3]
    int64_t* off = nullptr;     // [n + 1]
    int32_t* ent = nullptr;     // s: descends, ~s: paints the whole cell
    LevelIn in() const { return LevelIn{n, level, coord, off, ent}; }
    void free() {
        cudaFree(coord);
        cudaFree(off);
        cudaFree(ent);
        coord = nullptr;
        off = nullptr;
        ent = nullptr;
        n = 0;
    }
};

template <typename T>
cudaError_t dalloc(T** p, int64_t n) {
    *p = nullptr;
    return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (size_t)(n > 0 ? n : 1));
}

// The long cells of a level (lists longer than kChunkMinList) and the chunks of their children's lists (see
// chunk_firstref); *skip marks them for the level's other passes. Nothing when the level has none.
cudaError_t chunk_plan(const Level& L, DevBuf& buf, uint8_t** skip, std::vector<int64_t>* cells,
                       std::vector<ChunkWork>* work) {
    *skip = nullptr;
    cells->clear();
    work->clear();
    int64_t total = 0;  // entries of the whole level: no cell is long if they are few
    cudaError_t e = cudaMemcpy(&total, L.off + L.n, sizeof(int64_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess || total <= kChunkMinList) return e;
    uint8_t* sk = nullptr;
    int64_t *flag = nullptr, *out = nullptr;
    if ((e = buf.alloc(&sk, L.n)) != cudaSuccess || (e = buf.alloc(&flag, L.n)) != cudaSuccess) return e;
    flag_long<<<blocks_for(L.n, 256), 256>>>(L.in(), sk, flag);
    int64_t n_long = 0;
    if ((e = cudaGetLastError()) != cudaSuccess || (e = scan_i64(flag, L.n, &n_long)) != cudaSuccess) return e;
    if (n_long == 0) return cudaSuccess;
    if ((e = buf.alloc(&out, 3 * n_long)) != cudaSuccess) return e;
    gather_long<<<blocks_for(L.n, 256), 256>>>(L.in(), sk, flag, out);
    std::vector<int64_t> h((size_t)(3 * n_long));
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpy(h.data(), out, sizeof(int64_t) * h.size(), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return e;
    for (int64_t j = 0; j < n_long; ++j) {
        const int64_t i = h[(size_t)(3 * j)], b0 = h[(size_t)(3 * j + 1)], e0 = h[(size_t)(3 * j + 2)];
        cells->push_back(i);
        for (int k = 0; k < 8; ++k) {
            const int64_t fw = (int64_t)work->size();
            for (int64_t b = b0; b < e0; b += kChunk)
                work->push_back(ChunkWork{8 * i + k, b, std::min(e0, b + kChunk), fw, b == b0 ? 1 : 0});
        }
    }
    *skip = sk;
    return cudaSuccess;
}

// Expand one level: the eight child slots of each cell (*slot_out, handed to the caller: a leaf key, or
// kInternal | index in the next level) and the next level's refined cells with their lists.
cudaError_t expand(const Level& L, const StampDev& S, int32_t depth, double extent, double half, uint64_t** slot_out,
                   Level* next) {
    DevBuf buf;
    const int64_t nch = 8 * L.n;
    int32_t* fr;
    int64_t *cnt, *isint;
    uint64_t* slot;
    PCK(buf.alloc(&fr, nch));
    PCK(buf.alloc(&cnt, nch));
    PCK(buf.alloc(&isint, nch));
    PCK(dalloc(&slot, nch));
    *slot_out = slot;
    const LevelIn in = L.in();
    const bool split = L.n < kSplitCells;  // few cells: a warp per child
    // cells with long lists: a warp per chunk of a child's list (the passes below skip them)
    uint8_t* skip = nullptr;
    std::vector<int64_t> cells;
    std::vector<ChunkWork> work;
    PCK(chunk_plan(L, buf, &skip, &cells, &work));
    const int64_t nw = (int64_t)work.size(), nj = 8 * (int64_t)cells.size();
    ChunkWork* d_work = nullptr;
    int64_t *d_cells = nullptr, *chunk_cnt = nullptr, *npaint = nullptr;
    if (nw) {
        PCK(buf.alloc(&d_work, nw));
        PCK(buf.alloc(&d_cells, (int64_t)cells.size()));
        PCK(buf.alloc(&chunk_cnt, nw));
        PCK(buf.alloc(&npaint, nch));
        PCK(cudaMemcpy(d_work, work.data(), sizeof(ChunkWork) * (size_t)nw, cudaMemcpyHostToDevice));
        PCK(cudaMemcpy(d_cells, cells.data(), sizeof(int64_t) * cells.size(), cudaMemcpyHostToDevice));
        chunk_init<<<blocks_for(nj, 256), 256>>>(d_cells, nj, fr, cnt, npaint);
        chunk_firstref<<<blocks_for(nw, kWarpsPerBlock), 32 * kWarpsPerBlock>>>(in, S, depth, extent, half, d_work, nw, fr);
        chunk_count<<<blocks_for(nw, kWarpsPerBlock), 32 * kWarpsPerBlock>>>(in, S, extent, half, d_work, nw, fr, chunk_cnt,
                                                                             cnt, npaint);
        chunk_child_finish<<<blocks_for(nj, kWarpsPerBlock), 32 * kWarpsPerBlock>>>(in, S, extent, half, d_cells, nj, fr,
                                                                                   npaint, slot, cnt, isint);
    }
    if (split)
        expand_child_count<<<blocks_for(nch, kWarpsPerBlock), 32 * kWarpsPerBlock>>>(in, S, depth, extent, half, fr, slot,
                                                                                    cnt, isint, skip);
    else
        expand_parent_count<<<blocks_for(L.n, kWarpsPerBlock), 32 * kWarpsPerBlock>>>(in, S, depth, extent, half, fr,
                                                                                     slot, cnt, isint, skip);
    PCK(cudaGetLastError());
    int64_t n_ent = 0, n_next = 0;
    PCK(scan_i64(cnt, nch, &n_ent));
    PCK(scan_i64(isint, nch, &n_next));
    next->n = n_next;
    next->level = L.level + 1;
    if (n_next == 0) return cudaSuccess;  // no internal child: the slots are all leaf keys
    PCK(dalloc(&next->coord, 3 * n_next));
    PCK(dalloc(&next->off, n_next + 1));
    PCK(dalloc(&next->ent, n_ent));
    PCK(cudaMemcpy(next->off + n_next, &n_ent, sizeof(int64_t), cudaMemcpyHostToDevice));
    if (nw) {
        int64_t n_chunked = 0;
        PCK(scan_i64(chunk_cnt, nw, &n_chunked));  // per child: its list start plus the counts of earlier chunks
        chunk_write<<<blocks_for(nw, kWarpsPerBlock), 32 * kWarpsPerBlock>>>(in, S, extent, half, d_work, nw, fr, slot, cnt,
                                                                             isint, chunk_cnt, next->coord, next->off,
                                                                             next->ent);
    }
    if (split)
        expand_child_write<<<blocks_for(nch, kWarpsPerBlock), 32 * kWarpsPerBlock>>>(in, S, extent, half, fr, slot, cnt,
                                                                                    isint, next->coord, next->off,
                                                                                    next->ent, skip);
    else
        expand_parent_write<<<blocks_for(L.n, kWarpsPerBlock), 32 * kWarpsPerBlock>>>(in, S, extent, half, fr, slot,
                                                                                     cnt, isint, next->coord, next->off,
                                                                                     next->ent, skip);
    PCK(cudaGetLastError());
    return cudaDeviceSynchronize();
}

// Paint down from L (its arrays are freed on the way): slots and cell counts per level, until no refined cell is
// left, or up to level `stop` (that level's cells are then left unexpanded in *rest). With track, the cells of L
// are partitions 0 .. L.n - 1 and offs receives, per painted level, the first cell of each partition.
cudaError_t paint_down(Level L, const StampDev& S, int32_t depth, double extent, double half, int stop, bool track,
                       std::vector<uint64_t*>* slots, std::vector<int64_t>* ncell, Level* rest,
                       std::vector<int64_t*>* offs) {
    const int64_t nseg = L.n;
    int32_t* pid = nullptr;
    cudaError_t e = cudaSuccess;
    if (track && L.n > 0) {
        e = dalloc(&pid, L.n);
        if (e == cudaSuccess) iota32<<<blocks_for(L.n, 256), 256>>>(L.n, pid);
    }
    while (e == cudaSuccess && L.n > 0 && L.level != stop) {
        uint64_t* slot = nullptr;
        Level next;
        e = expand(L, S, depth, extent, half, &slot, &next);
        if (slot) {
            slots->push_back(slot);
            ncell->push_back(L.n);
        }
        if (e == cudaSuccess && track) {
            int64_t* off = nullptr;
            e = dalloc(&off, nseg + 1);
            if (e == cudaSuccess) {
                offs->push_back(off);
                seg_offsets<<<blocks_for(nseg + 1, 256), 256>>>(L.n, pid, nseg, off);
                int32_t* pid_next = nullptr;
                if (next.n > 0 && (e = dalloc(&pid_next, next.n)) == cudaSuccess)
                    pid_propagate<<<blocks_for(8 * L.n, 256), 256>>>(L.n, slot, pid, pid_next);
                if (e == cudaSuccess) e = cudaGetLastError();
                cudaFree(pid);
                pid = pid_next;
            }
        }
        L.free();
        L = next;
        if (e != cudaSuccess) L.free();
    }
    cudaFree(pid);
    if (e == cudaSuccess && L.n > 0 && L.level == stop) {
        *rest = L;
    } else {
        L.free();
        rest->n = 0;
        rest->level = stop;
    }
    return e == cudaSuccess ? cudaDeviceSynchronize() : e;
}

}  // namespace

// What the painter keeps of a painted canvas for appends: the level-P cells (Morton codes and stamp lists) and
// the slots of every level from P down, with each partition's first cell per level.
struct PaintCache {
    int32_t depth = 0;
    double extent = 0.0;
    int64_t n_stamps = 0;       // stamps painted
    int64_t nP = 0;             // refined cells at the partition level
    uint64_t* code = nullptr;   // [nP] Morton codes (ascending)
    int64_t* lst_off = nullptr; // [nP + 1]
    int32_t* lst_ent = nullptr; // their stamp lists
    std::vector<uint64_t*> slots;  // levels P, P + 1, ...
    std::vector<int64_t> ncell;
    std::vector<int64_t*> off;     // per level: [nP + 1] first cell of each partition
};

void paint_cache_free(PaintCache* c) {
    if (!c) return;
    cudaFree(c->code);
    cudaFree(c->lst_off);
    cudaFree(c->lst_ent);
    for (auto* p : c->slots) cudaFree(p);
    for (auto* p : c->off) cudaFree(p);
    delete c;
}

namespace {

constexpr int kPartLevel = 5;  // partition level: up to 32,768 partitions

void free_all(std::vector<uint64_t*>& v) {
    for (auto* p : v) cudaFree(p);
    v.clear();
}
void free_all(std::vector<int64_t*>& v) {
    for (auto* p : v) cudaFree(p);
    v.clear();
}

// The root with the stamps [0, n) that touch the canvas, in order.
cudaError_t root_level(const StampDev& S, int64_t n, double extent, double half, Level* root) {
    DevBuf buf;
    int64_t *flag, *flag_scan, n_root = 0;
    PCK(buf.alloc(&flag, n));
    PCK(buf.alloc(&flag_scan, n));
    if (n > 0) {
        root_flags<<<blocks_for(n, 256), 256>>>(S, n, extent, half, flag);
        PCK(cudaGetLastError());
        PCK(cudaMemcpy(flag_scan, flag, sizeof(int64_t) * (size_t)n, cudaMemcpyDeviceToDevice));
        PCK(scan_i64(flag_scan, n, &n_root));
    }
    root->n = 1;
    root->level = 0;
    PCK(dalloc(&root->coord, 3));
    PCK(dalloc(&root->off, 2));
    PCK(dalloc(&root->ent, n_root));
    PCK(cudaMemset(root->coord, 0, 3 * sizeof(uint32_t)));
    const int64_t off0[2] = {0, n_root};
    PCK(cudaMemcpy(root->off, off0, sizeof(off0), cudaMemcpyHostToDevice));
    if (n > 0) {
        root_write<<<blocks_for(n, 256), 256>>>(n, flag_scan, flag, root->ent);
        PCK(cudaGetLastError());
    }
    return cudaDeviceSynchronize();
}

// Per-level partition offsets and slots of the appended canvas, from the kept subtrees (reuse[p] >= 0) and the
// repainted ones (rep[p] >= 0).
cudaError_t assemble(int64_t n_part, const int32_t* reuse, const int32_t* rep, const PaintCache& old,
                     const std::vector<uint64_t*>& slots_r, const std::vector<int64_t*>& offs_r,
                     std::vector<uint64_t*>* slots, std::vector<int64_t>* ncell, std::vector<int64_t*>* offs) {
    DevBuf buf;
    int64_t* cnt;
    PCK(buf.alloc(&cnt, n_part));
    const size_t depth_max = std::max(old.slots.size(), slots_r.size());
    for (size_t d = 0; d < depth_max; ++d) {
        part_counts<<<blocks_for(n_part, 256), 256>>>(n_part, reuse, rep, d < old.off.size() ? old.off[d] : nullptr,
                                                      d < offs_r.size() ? offs_r[d] : nullptr, cnt);
        PCK(cudaGetLastError());
        int64_t* off;
        PCK(dalloc(&off, n_part + 1));
        offs->push_back(off);
        PCK(cudaMemcpy(off, cnt, sizeof(int64_t) * (size_t)n_part, cudaMemcpyDeviceToDevice));
        int64_t total = 0;
        PCK(scan_i64(off, n_part, &total));
        PCK(cudaMemcpy(off + n_part, &total, sizeof(int64_t), cudaMemcpyHostToDevice));
        if (total == 0) {
            cudaFree(off);
            offs->pop_back();
            break;
        }
        ncell->push_back(total);
    }
    for (size_t d = 0; d < ncell->size(); ++d) {
        uint64_t* slot;
        PCK(dalloc(&slot, 8 * (*ncell)[d]));
        slots->push_back(slot);
        const bool last = d + 1 == ncell->size();
        assemble_level<<<blocks_for(8 * (*ncell)[d], 256), 256>>>(
            (*ncell)[d], n_part, (*offs)[d], last ? nullptr : (*offs)[d + 1], reuse, rep,
            d < old.slots.size() ? old.slots[d] : nullptr, d < old.off.size() ? old.off[d] : nullptr,
            d + 1 < old.off.size() ? old.off[d + 1] : nullptr, d < slots_r.size() ? slots_r[d] : nullptr,
            d < offs_r.size() ? offs_r[d] : nullptr, d + 1 < offs_r.size() ? offs_r[d + 1] : nullptr, slot);
        PCK(cudaGetLastError());
    }
    return cudaDeviceSynchronize();
}

}  // namespace

cudaError_t paint_pools(int32_t depth, double extent, const double* d_c, const double* d_r, const float4* d_rgba,
                        int64_t n, PaintCache** cache, int32_t** d_nodes_out, uint2** d_leaves_out, int64_t* n_rec_out,
                        int64_t* n_leaf_out, std::vector<int64_t>* level_begin, int64_t* wrap_out,
                        int32_t* n_wrap_out) {
    const double half = 0.5 * extent;
    PaintCache* old = *cache;
    *cache = nullptr;
    // an append: the same canvas, and the stamps the cache was painted with come first in the table
    const bool append = old && old->depth == depth && old->extent == extent && old->n_stamps <= n;
    DevBuf buf;
    // squared radii and target depths (the host painter's integer loop, in the same FP64 operations)
    double* d_r2;
    int32_t* d_kt;
    cudaError_t e = buf.alloc(&d_r2, n);
    if (e == cudaSuccess) e = buf.alloc(&d_kt, n);
    if (e == cudaSuccess && n > 0) {
        stamp_prep<<<blocks_for(n, 256), 256>>>(d_r, n, depth, extent, d_r2, d_kt);
        e = cudaGetLastError();
    }
    const StampDev S{d_c, d_r2, d_kt, d_rgba};
    // levels 0 .. P - 1 from the root (always painted: every stamp reaches the root's list)
    std::vector<uint64_t*> slots_top, slots_bot, slots_r;
    std::vector<int64_t> ncell_top, ncell_bot, ncell_r;
    std::vector<int64_t*> offs_bot, offs_r;
    Level root, partP, rep_lvl, unused;
    PaintCache* nc = nullptr;
    if (e == cudaSuccess) e = root_level(S, n, extent, half, &root);
    if (e == cudaSuccess) e = paint_down(root, S, depth, extent, half, kPartLevel, false, &slots_top, &ncell_top, &partP, nullptr);
    else root.free();
    if (e == cudaSuccess) {
        nc = new PaintCache();
        nc->depth = depth;
        nc->extent = extent;
        nc->n_stamps = n;
        nc->nP = partP.n;
        e = dalloc(&nc->code, partP.n);
        if (e == cudaSuccess && partP.n > 0) {
            morton_codes<<<blocks_for(partP.n, 256), 256>>>(partP.n, partP.coord, kPartLevel, nc->code);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess && !append) {
        // a full paint: every partition painted, a copy of their lists kept
        Level start = partP;
        int64_t* keep_off = nullptr;
        int32_t* keep_ent = nullptr;
        e = dalloc(&keep_off, partP.n + 1);
        if (e == cudaSuccess) e = dalloc(&keep_ent, 1);
        if (e == cudaSuccess && partP.n > 0) {
            int64_t n_ent = 0;
            e = cudaMemcpy(&n_ent, partP.off + partP.n, sizeof(int64_t), cudaMemcpyDeviceToHost);
            cudaFree(keep_ent);
            keep_ent = nullptr;
            if (e == cudaSuccess) e = dalloc(&keep_ent, n_ent);
            if (e == cudaSuccess)
                e = cudaMemcpy(keep_ent, partP.ent, sizeof(int32_t) * (size_t)n_ent, cudaMemcpyDeviceToDevice);
            if (e == cudaSuccess)
                e = cudaMemcpy(keep_off, partP.off, sizeof(int64_t) * (size_t)(partP.n + 1), cudaMemcpyDeviceToDevice);
        }
        nc->lst_off = keep_off;
        nc->lst_ent = keep_ent;
        if (e == cudaSuccess)
            e = paint_down(start, S, depth, extent, half, -1, true, &slots_bot, &ncell_bot, &unused, &offs_bot);
        else
            start.free();
        partP = Level();
    } else if (e == cudaSuccess) {
        // an append: keep the partitions whose cell and stamp list are unchanged, paint the others again
        int32_t *reuse = nullptr, *rep = nullptr, *sel = nullptr;
        int64_t* len = nullptr;
        const int64_t np = partP.n;
        std::vector<int32_t> h_reuse((size_t)np), h_rep((size_t)np, -1), h_sel;
        e = buf.alloc(&reuse, np);
        if (e == cudaSuccess && np > 0) {
            match_partitions<<<blocks_for(32 * np, 256), 256>>>(np, partP.coord, partP.off, partP.ent, old->nP, old->code,
                                                                old->lst_off, old->lst_ent, kPartLevel, reuse);
            e = cudaGetLastError();
            if (e == cudaSuccess)
                e = cudaMemcpy(h_reuse.data(), reuse, sizeof(int32_t) * (size_t)np, cudaMemcpyDeviceToHost);
        }
        for (int64_t p = 0; p < np; ++p)
            if (h_reuse[(size_t)p] < 0) {
                h_rep[(size_t)p] = (int32_t)h_sel.size();
                h_sel.push_back((int32_t)p);
            }
        const int64_t m = (int64_t)h_sel.size();
        if (e == cudaSuccess) e = buf.alloc(&rep, np);
        if (e == cudaSuccess) e = buf.alloc(&sel, m);
        if (e == cudaSuccess) e = buf.alloc(&len, m + 1);
        if (e == cudaSuccess && np > 0) e = cudaMemcpy(rep, h_rep.data(), sizeof(int32_t) * (size_t)np, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && m > 0) e = cudaMemcpy(sel, h_sel.data(), sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice);
        // the repainted partitions as one level
        rep_lvl.n = m;
        rep_lvl.level = kPartLevel;
        if (e == cudaSuccess && m > 0) {
            list_lengths<<<blocks_for(m, 256), 256>>>(m, sel, partP.off, len);
            int64_t n_ent = 0;
            e = scan_i64(len, m, &n_ent);
            if (e == cudaSuccess) e = cudaMemcpy(len + m, &n_ent, sizeof(int64_t), cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = dalloc(&rep_lvl.coord, 3 * m);
            if (e == cudaSuccess) e = dalloc(&rep_lvl.off, m + 1);
            if (e == cudaSuccess) e = dalloc(&rep_lvl.ent, n_ent);
            if (e == cudaSuccess) {
                gather_cells<<<blocks_for(32 * m, 256), 256>>>(m, sel, partP.coord, partP.off, partP.ent, len,
                                                               rep_lvl.coord, rep_lvl.off, rep_lvl.ent);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess)
                e = cudaMemcpy(rep_lvl.off + m, &n_ent, sizeof(int64_t), cudaMemcpyHostToDevice);
        }
        if (e == cudaSuccess)
            e = paint_down(rep_lvl, S, depth, extent, half, -1, true, &slots_r, &ncell_r, &unused, &offs_r);
        else
            rep_lvl.free();
        if (e == cudaSuccess) e = assemble(np, reuse, rep, *old, slots_r, offs_r, &slots_bot, &ncell_bot, &offs_bot);
        free_all(slots_r);
        free_all(offs_r);
        // the new level-P lists are kept
        nc->lst_off = partP.off;
        nc->lst_ent = partP.ent;
        cudaFree(partP.coord);
        partP = Level();
    }
    paint_cache_free(old);
    if (e == cudaSuccess) {
        std::vector<uint64_t*> all(slots_top);
        all.insert(all.end(), slots_bot.begin(), slots_bot.end());
        std::vector<int64_t> cells(ncell_top);
        cells.insert(cells.end(), ncell_bot.begin(), ncell_bot.end());
        e = finish_pools(all, cells, d_nodes_out, d_leaves_out, n_rec_out, n_leaf_out, level_begin, wrap_out, n_wrap_out);
    }
    free_all(slots_top);
    partP.free();
    if (e == cudaSuccess) {
        nc->slots = slots_bot;
        nc->ncell = ncell_bot;
        nc->off = offs_bot;
        *cache = nc;
    } else {
        free_all(slots_bot);
        free_all(offs_bot);
        paint_cache_free(nc);
    }
    return e;
}

}  // namespace canvox
