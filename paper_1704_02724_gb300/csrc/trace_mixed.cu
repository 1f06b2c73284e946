// Mixed-precision persistent ray caster for deep sparse octrees (sm_103a).
//
// One lane traces one ray (Sec. 6 of the paper): from the FP64 eye (Sec. 6.1)
// leaf by leaf through the octree, compositing front to back, until the
// transmittance drops below t_min or the ray leaves the canvas (Sec. 6.2).
//
// Cells are addressed by exact integer coordinates (level L, c in [0, 2^L)^3).
// Crossing a face moves c by one on the exit axis; the lowest common ancestor
// of the old and new cell is L - bitlength(c_old ^ c_new). The new leaf is
// found from the neighbouring cell: a sibling in the same record, else the
// slot the parent's neighbour link names (the neighbour graph of Sec. 4.1.1,
// built at upload), or, in the stack traversal, the ancestor's record kept on
// a per-lane stack of records by level; then a descent while the cell is
// internal. The integer bits fix the path down to the old cell's level; only
// deeper levels need the ray's position.
//
// Precision (Sec. 6.1-6.3). The ray is evaluated inside a local frame, a cell
// of level f <= L at most K levels above the leaf, in frame units:
//     t'(P') = P' inv_d + nod_f,   t' = (t - t_f) / S_f,
// where P' is a cell plane in frame units (an exact dyadic FP32 value), t_f the
// FP64 ray parameter where the frame was entered and S_f its size. This is the
// paper's cell-local frame (origin at a cell, unit size) widened from one cell
// to a subtree. The frame is re-anchored in FP64 whenever the ray leaves it, so
// the drift of Sec. 6.3 (e0 + 7.5 eps L) does not accumulate across frames:
// on a frame exit to the coarsest frame that holds the new leaf, on a descent
// more than K levels below the frame to the frame depth - K (the deepest one
// the canvas can need), so that a ray entering a deep region rebases once; a
// ray that starts at the eye's leaf takes that frame from the start.
// inv_d and nod_f are each kept as two FP32 words. Decisions (which face of the
// leaf the ray leaves by, which side of a mid-plane it is on) are screened in
// plain FP32 with a proven margin, and taken in FP64 from the exact planes when
// the screen cannot decide (the ray passes within about 2^-22 frame units of an
// edge or a plane: a few steps in a hundred thousand). The time of the exit
// face, which sets the segment length, is a double-float: an unevaluated sum
// hi + lo of two FP32 words formed with error-free transformations (Dekker's
// product by fma, Knuth's two-sum), good to about 2^-44 |inv_d| frame units.
// A boundary between leaves of different value moves the pixel by at most
// 2 T max(sigma) |dt|; each ray carries a budget for these bounds, and a
// boundary whose bound would exceed it is recomputed in FP64.
//
// Compositing (emission-absorption reading of Sec. 6.2): per segment of signed
// length l in a leaf (sigma, rgb): a = 1 - exp(-sigma l), C += T a rgb,
// T *= 1 - a, with a compensated (Kahan) FP32 sum for C and the transmittance
// kept as a running product (one rounding per leaf, unbiased).
//
// The per-lane counters of slot reads, leaf loads and record loads (the
// algorithmic bytes of a render) are a template option: a render that does
// not report them runs without them.
#include <cuda_fp16.h>

#include "canvox_internal.cuh"

namespace canvox {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr float kEpsDF = 5.684341886080802e-14f;   // 2^-44: double-float crossing-time bound per |inv_d|
constexpr float kEpsDF2 = 1.1368683772161603e-13f; // 2^-43 = 2 * 2^-44: factor 2 of the colour bound
constexpr int kMaxFrameBits = 22;                   // a frame spans at most 22 levels (exact FP32 planes)
constexpr float kEps21 = 4.76837158203125e-07f;     // 2^-21
constexpr float kEps22 = 2.384185791015625e-07f;    // 2^-22
constexpr float kEps41 = 4.547473508864641e-13f;    // 2^-41
constexpr float kBigF = 1.0e37f;                    // stands for the time of a face the ray never meets (d_a = 0)

// Resident 256-thread blocks per SM the register allocation must allow (occupancy knob).
#ifndef CANVOX_MIN_BLOCKS
#define CANVOX_MIN_BLOCKS 4
#endif

__device__ __forceinline__ double pow2d(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }
// IEEE binary16 bits -> float (exact: every half is a float).
__device__ __forceinline__ float half_bits_to_float(unsigned h) { return __half2float(__ushort_as_half((unsigned short)h)); }
__device__ __forceinline__ float hsig(uint2 v) { return half_bits_to_float(v.y >> 16); }
__device__ __forceinline__ float hlo(unsigned w) { return half_bits_to_float(w & 0xFFFFu); }
__device__ __forceinline__ float hhi(unsigned w) { return half_bits_to_float(w >> 16); }
// (float)x for x < 2^23, exactly, without a conversion instruction.
__device__ __forceinline__ float small_uint_to_float(uint32_t x) {
    return __fsub_rn(__int_as_float((int)(0x4B000000u | x)), 8388608.0f);
}

// x[a] for a runtime axis without indexing an array (which would put it in local memory).
template <typename V>
__device__ __forceinline__ V pick(int a, V x0, V x1, V x2) { return a == 0 ? x0 : (a == 1 ? x1 : x2); }

extern __shared__ int32_t s_nodes[];  // copy of the tree's first records (kernel instance with kSmem)

// Child slot k of record rec: from the shared-memory copy of the tree's breadth-first prefix when the
// kernel keeps one and the record is in it (records [0, n_smem)), else through the read-only data cache.
template <bool kSmem>
__device__ __forceinline__ int32_t load_slot(const Tree& T, int32_t n_smem, int32_t rec, int k) {
    if (kSmem && rec < n_smem) return s_nodes[rec * 8 + k];
    return __ldg(T.nodes + (int64_t)rec * 8 + k);
}
// Value of the leaf in slot k of record rec (slot value v < 0).
__device__ __forceinline__ uint2 load_leaf(const Tree& T, int32_t rec, int k, int32_t v) {
    return __ldg(T.leaves + leaf_index(T, rec, k, v));
}

__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

// t'(P) = P (ih + il) + (nh + nl) as hi + lo. P is exact; the product error
// comes from one fma and the sum error from Knuth's two-sum, both exact.
__device__ __forceinline__ void df_cross(float P, float ih, float il, float nh, float nl, float& hi, float& lo) {
    const float p = __fmul_rn(P, ih);
    const float pe = __fmaf_rn(P, ih, -p);
    const float s = __fadd_rn(p, nh);
    const float v = __fsub_rn(s, p);
    const float se = __fadd_rn(__fsub_rn(p, __fsub_rn(s, v)), __fsub_rn(nh, v));
    const float t = __fadd_rn(__fadd_rn(pe, se), __fmaf_rn(P, il, nl));
    hi = __fadd_rn(s, t);
    lo = __fsub_rn(t, __fsub_rn(hi, s));
}

constexpr int kBlock = 256;

// FP64 state, output address and rare counters of a lane: read only by rebases,
// near-ties, start-up and the final write, so it lives in shared memory.
struct Cold {
    double inv64[3], nod64[3];  // t(P) = P inv + nod; axis with d = 0: inv = 0, nod = o
    double tf;                  // FP64 ray parameter at the frame origin
    double invS;                // 1 / frame size
    uint32_t pix;               // output pixel within the view (below width * height < 2^31)
    int32_t view;
    uint32_t n_rays, n_steps, n_f64, n_rebase;
};
static_assert(sizeof(Cold) == 88, "per-lane shared record: 88 bytes keeps four blocks within the 132 KB carve-out");

struct Ray {
    Cold* k;
    float ih[3], il[3];         // inv_d as two FP32 words; for d_a = 0 the frame-local position, low word in ih
    float nh[3], nl[3];         // frame-local nod as two FP32 words; for d_a = 0: kBigF and 0, so that the far
                                // face of that axis evaluates to the time kBigF with no test
    float sf, sf_eps;           // frame size, frame size * 2^-43
    float gscr;                 // 2^-41 max (|ih_a| + |nh_a|) over the axes with d_a != 0: the screens' margin term
    float cur_hi, cur_lo;       // frame-local parameter of the current leaf's entry
    float2* acc;  // shared, stride kBlock: (sum, Kahan term) of the colour channels 0, 1, 2
    float* err;   // shared: colour-error bound spent so far (the budget of the FP32 boundaries)
    float T;
    uint32_t c[3];
    int32_t L, f;
    uint32_t dpos, zmask;
    uint2 val;
    int32_t pr;   // record holding the current leaf's slot (neighbour-link traversal)
    uint32_t kc;  // child index of the current leaf in pr
    int32_t steps;
    // counters, summed over every ray the lane traces
    uint32_t n_reads, n_leaf, n_rec;
};

__device__ __forceinline__ bool is_zero(const Ray& r, int a) { return (r.zmask >> a) & 1u; }
#define ACC(r, i) ((r).acc[(i) * kBlock])
#define ERR(r) (*(r).err)

// Ray on the high side of the global plane x_a = M just after parameter t (FP64).
__device__ __forceinline__ uint32_t high64(const Ray& r, int a, double M, double t) {
    if (is_zero(r, a)) return r.k->nod64[a] >= M;
    const double tm = fma(M, r.k->inv64[a], r.k->nod64[a]);
    return r.k->inv64[a] > 0.0 ? (tm <= t) : (tm > t);
}

// FP64 crossing time of the face (c + s) of a level-L cell on axis a (exact plane).
__device__ __forceinline__ double face_t64(const Ray& r, const Tree& T, int a, uint32_t cs, int L) {
    const double P = fma((double)cs, T.extent * pow2d(-L), -T.half);
    return fma(P, r.k->inv64[a], r.k->nod64[a]);
}

__device__ __forceinline__ void split_local(const Ray& r, double t, float& hi, float& lo) {
    const double tl = (t - r.k->tf) * r.k->invS;
    hi = (float)tl;
    lo = (float)(tl - (double)hi);
}

// Exit face of the level-L leaf c by the FP64 crossing times of its exact far planes (ties to the lowest
// axis), and that time as a frame-local double-float. Taken on a few leaf steps in a hundred thousand (a
// ray within about 2^-22 frame units of an edge), so it is kept out of line: its FP64 code then does not
// weigh on the register allocation of the step loop.
struct Exit64 {
    double t;
    float hi, lo;
    int ax;
};
__device__ __noinline__ Exit64 exit_face64(Cold* k, uint32_t zmask, uint32_t dpos, uint32_t c0, uint32_t c1, uint32_t c2,
                                           int L, double extent, double half) {
    Exit64 e;
    e.t = __longlong_as_double(0x7FF0000000000000ll);
    e.ax = 0;
    const double w = extent * pow2d(-L);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if ((zmask >> a) & 1u) continue;
        const uint32_t cs = (a == 0 ? c0 : (a == 1 ? c1 : c2)) + ((dpos >> a) & 1u);
        const double ta = fma(fma((double)cs, w, -half), k->inv64[a], k->nod64[a]);
        if (ta < e.t) {
            e.t = ta;
            e.ax = a;
        }
    }
    const double tl = (e.t - k->tf) * k->invS;
    e.hi = (float)tl;
    e.lo = (float)(tl - (double)e.hi);
    k->n_f64 += 1;
    return e;
}

// Enter the frame at level r.f that holds the cell (r.L, r.c); t = FP64 parameter of the entry.
__device__ __forceinline__ void set_frame(Ray& r, const Tree& T, double inv_extent, double t) {
    r.k->tf = t;
    const int sh = r.L - r.f;
    const double Sf = T.extent * pow2d(-r.f);
    r.k->invS = pow2d(r.f) * inv_extent;
    float g = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double Fmin = fma((double)(r.c[a] >> sh), Sf, -T.half);
        if (is_zero(r, a)) {
            const double n = (r.k->nod64[a] - Fmin) * r.k->invS;
            r.il[a] = (float)n;
            r.ih[a] = (float)(n - (double)r.il[a]);
            r.nh[a] = kBigF;
            r.nl[a] = 0.0f;
        } else {
            const double n = (fma(Fmin, r.k->inv64[a], r.k->nod64[a]) - t) * r.k->invS;
            r.nh[a] = (float)n;
            r.nl[a] = (float)(n - (double)r.nh[a]);
            g = fmaxf(g, __fadd_rn(fabsf(r.ih[a]), fabsf(r.nh[a])));
        }
    }
    r.gscr = __fmul_rn(kEps41, g);
    r.sf = (float)Sf;
    r.sf_eps = r.sf * kEpsDF2;
    r.cur_hi = 0.0f;
    r.cur_lo = 0.0f;
    r.k->n_rebase += 1;
}

// Composite the current leaf over [cursor, te]. The length is not clamped at
// zero: a boundary can land slightly before the cursor (within its error
// bound), and only the signed lengths of consecutive segments telescope, so a
// boundary between two leaves of equal value then costs nothing.
__device__ __forceinline__ void kahan_add2(float2& sc, float x) { kahan_add(sc.x, sc.y, x); }

__device__ __forceinline__ void composite(Ray& r, float teh, float tel) {
    const float ell = ((teh - r.cur_hi) + (tel - r.cur_lo)) * r.sf;
    if (r.val.y >> 16) {
        const float s = hsig(r.val);
        const float em = expm1f(-s * ell);  // -a
        const float w = -r.T * em;
        float2 c0 = ACC(r, 0), c1 = ACC(r, 1), c2 = ACC(r, 2);
        kahan_add2(c0, w * hlo(r.val.x));
        kahan_add2(c1, w * hhi(r.val.x));
        kahan_add2(c2, w * hlo(r.val.y));
        ACC(r, 0) = c0;
        ACC(r, 1) = c1;
        ACC(r, 2) = c2;
        r.T = __fmaf_rn(r.T, em, r.T);  // T (1 - a)
    }
}

__device__ __forceinline__ void finish(Ray& r, const MixedParams& P) {
    const View& V = P.views[r.k->view];
    float4 o;
    o.x = ACC(r, 0).x + r.T * V.bg[0];
    o.y = ACC(r, 1).x + r.T * V.bg[1];
    o.z = ACC(r, 2).x + r.T * V.bg[2];
    o.w = 1.0f - r.T;
    const int64_t pix = V.out_offset + (int64_t)r.k->pix;
    P.out[pix] = o;
    if (P.step_count) P.step_count[pix] = r.steps;
    r.k->n_rays += 1;
    r.k->n_steps += (uint32_t)r.steps;
}

// Child bit on axis a of the cell at level `lev` with coordinate cc, for the ray
// just after the frame-local time (th, tl) (a double-float whose own error is
// at most margin_t). Screened in plain FP32: the mid-plane time
//     F = fl(fl(Mp ih + nh) + fl(Mp il + nl))        (Mp <= 1: a frame plane)
// is within 2^-23 |F| + 2^-47 (|ih| + |nh|) of the exact time, and the
// difference D = fl(fl(F - th) - tl) within 2^-23 (|F| + |th| + |D|) more.
// The side is the sign of D when
//     |D| > fl(2^-21 |F| + base),   base = fl(2^-21 |th| + fl(gscr + margin_t))
// (the caller forms base once per leaf step). Its 2^-21 is twice the 2^-22 that
// the error terms in |F| and |th| need, which leaves room for the three roundings
// of the screen and for the 2^-23 |D| term; the frame's gscr = 2^-41 max_b
// (|ih_b| + |nh_b|) covers the 2^-47 term 64 times over. Otherwise, and for
// frames deeper than 22 levels, it returns kUndecided: the caller decides in
// FP64 (side64), once per level for all the sides left open.
constexpr uint32_t kUndecided = 2u;
__device__ __forceinline__ uint32_t child_side(const Ray& r, int a, uint32_t cc, int lev, float th, float tl,
                                               float base) {
    if (lev - r.f < kMaxFrameBits) {
        const uint32_t rel = cc & ((1u << (lev - r.f)) - 1u);
        const float Mp = small_uint_to_float(2u * rel + 1u) * pow2f(-(lev + 1 - r.f));
        if (is_zero(r, a)) {
            const float dm = __fadd_rn(__fsub_rn(r.il[a], Mp), r.ih[a]);
            if (fabsf(dm) > kEpsDF) return dm >= 0.0f;
        } else {
            const float F = __fadd_rn(__fmaf_rn(Mp, r.ih[a], r.nh[a]), __fmaf_rn(Mp, r.il[a], r.nl[a]));
            const float D = __fsub_rn(__fsub_rn(F, th), tl);
            if (fabsf(D) > __fmaf_rn(kEps21, fabsf(F), base)) return r.ih[a] > 0.0f ? (D <= 0.0f) : (D > 0.0f);
        }
    }
    return kUndecided;
}

// FP64 side of the mid-plane of cell cc (level lev) on axis a just after FP64 time t.
__device__ __forceinline__ uint32_t side64(const Ray& r, const Tree& T, int a, uint32_t cc, int lev, double t) {
    const double M = fma((double)(2u * cc + 1u), T.extent * pow2d(-(lev + 1)), -T.half);
    return high64(r, a, M, t);
}

// Frame level for a leaf at level L that has descended past its frame, and for a ray's first frame at the eye's
// leaf: the level depth - K that holds the canvas's deepest leaves within K levels, kept within [L - K, L].
__device__ __forceinline__ int deep_frame(int L, int depth, int K) { return max(L - K, min(max(0, depth - K), L)); }

// Start ray g of the launch. Returns true if it has a leaf to step from.
template <bool kSmem, bool kRopes, bool kCount>
__device__ bool ray_init(Ray& r, const MixedParams& P, double inv_extent, unsigned long long g, int32_t* stk) {
    const Tree& T = P.tree;
    g += (unsigned long long)P.ray_base;
    int lo = 0, hi = P.n_views - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((unsigned long long)P.views[mid].ray_begin <= g) lo = mid;
        else hi = mid - 1;
    }
    const View& V = P.views[lo];
    const long long local = (long long)g - V.ray_begin;
    const unsigned tile = (unsigned)(local >> 5);  // tiles of one view fit 32 bits (width, height < 2^31)
    const int lane = (int)(local & 31);
    const unsigned ty = tile / (unsigned)V.tiles_x;
    const int wl = V.tile_wl;
    const int i = ((int)(tile - ty * (unsigned)V.tiles_x) << wl) + (lane & ((1 << wl) - 1));
    const int j = (int)ty * (32 >> wl) + (lane >> wl);
    if (i >= V.width || j >= V.height) return false;  // padding lane of a ragged tile
    r.k->view = lo;
    r.k->pix = (uint32_t)j * (uint32_t)V.width + (uint32_t)i;
    ACC(r, 0) = ACC(r, 1) = ACC(r, 2) = make_float2(0.0f, 0.0f);
    r.T = 1.0f;
    ERR(r) = 0.0f;
    r.steps = 0;
    // pixel-centre ray in FP64 (Sec. 6.1)
    double d[3];
    pixel_ray(V, i, j, d);
    r.dpos = 0;
    r.zmask = 0;
    double t0 = 0.0, t1 = __longlong_as_double(0x7FF0000000000000ll);
    bool miss = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double da = d[a];
        const double o = V.eye[a];
        if (da != 0.0) {
            r.k->inv64[a] = 1.0 / da;
            r.k->nod64[a] = -o * r.k->inv64[a];
            r.ih[a] = (float)r.k->inv64[a];
            r.il[a] = (float)(r.k->inv64[a] - (double)r.ih[a]);
            if (da > 0.0) r.dpos |= 1u << a;
            const double ta = fma(-T.half, r.k->inv64[a], r.k->nod64[a]);
            const double tb = fma(T.half, r.k->inv64[a], r.k->nod64[a]);
            t0 = fmax(t0, da > 0.0 ? ta : tb);
            t1 = fmin(t1, da > 0.0 ? tb : ta);
        } else {
            r.k->inv64[a] = 0.0;
            r.k->nod64[a] = o;
            r.ih[a] = 0.0f;
            r.il[a] = 0.0f;
            r.zmask |= 1u << a;
            if (!(o >= -T.half && o < T.half)) miss = true;
        }
    }
    if (miss || !(t0 < t1)) {
        finish(r, P);
        return false;
    }
    const EyePath& E = P.eye[r.k->view];
    if (E.len > 0 && t0 == 0.0) {
        // the eye's leaf, located once for the view
        r.L = E.len;
        if (kRopes) {
            r.pr = E.rec[E.len - 1];
            r.kc = (E.c[0] & 1u) | ((E.c[1] & 1u) << 1) | ((E.c[2] & 1u) << 2);
        } else {
            for (int l = 0; l < E.len; ++l) stk[l] = E.rec[l];
        }
        r.c[0] = E.c[0];
        r.c[1] = E.c[1];
        r.c[2] = E.c[2];
        r.val = E.val;
        if (kCount) r.n_reads += r.L;
        if (kCount) r.n_leaf += (uint32_t)E.stored;
        r.steps = 1;
        // the frame a descent would settle in (depth - K, within [L - K, L]): rays that start in a deep subtree
        // do not rebase again on their first descent past the eye's frame
        r.f = deep_frame(r.L, T.depth, P.frame_levels);
        set_frame(r, T, inv_extent, t0);
        return true;
    }
    // locate the leaf that holds r(t0+) from the root, in double-float frames (frame time 0)
    r.c[0] = r.c[1] = r.c[2] = 0u;
    r.L = 0;
    r.f = 0;
    set_frame(r, T, inv_extent, t0);
    int lev = 0;
    int32_t rec = 0;
    int32_t slot;
    stk[0] = 0;
    for (;;) {
        if (lev - r.f >= kMaxFrameBits) {
            // planes of the next level need more than 22 bits in this frame: re-anchor at this cell
            r.L = lev;
            r.f = lev;
            set_frame(r, T, inv_extent, t0);
        }
        uint32_t b3[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) b3[a] = child_side(r, a, r.c[a], lev, 0.0f, 0.0f, r.gscr);
        if (b3[0] == kUndecided || b3[1] == kUndecided || b3[2] == kUndecided) {
#pragma unroll
            for (int a = 0; a < 3; ++a)
                if (b3[a] == kUndecided) b3[a] = side64(r, T, a, r.c[a], lev, t0);
        }
        int k = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            r.c[a] = 2u * r.c[a] + b3[a];
            k |= (int)b3[a] << a;
        }
        slot = load_slot<kSmem>(T, P.smem_records, rec, k);
        if (kCount) r.n_rec += 1;
        if (slot > 0) {
            ++lev;
            if (!kRopes) stk[lev] = slot;
            rec = slot;
        } else {
            r.pr = rec;
            r.kc = (uint32_t)k;
            break;
        }
    }
    r.L = lev + 1;
    if (kCount) r.n_reads += r.L;
    if (slot < 0) {
        r.val = load_leaf(T, rec, (int)r.kc, slot);
        if (kCount) r.n_leaf += 1;
    } else {
        r.val = make_uint2(0u, 0u);
    }
    r.steps = 1;
    if (r.L - r.f > P.frame_levels) {
        r.f = deep_frame(r.L, T.depth, P.frame_levels);
        set_frame(r, T, inv_extent, t0);
    }
    return true;
}

// One leaf step. Returns false once the ray is finished (its pixel written).
template <bool kSmem, bool kRopes, bool kCount>
__device__ bool ray_step(Ray& r, const MixedParams& P, double inv_extent, int32_t* stk) {
    const Tree& T = P.tree;
    // 1. exit of the current leaf: the far face on each axis is the plane P_a (frame units, exact)
    const int kf = r.L - r.f;
    const float sc = pow2f(-kf);
    const uint32_t fmask = (1u << kf) - 1u;
    const float P0 = small_uint_to_float((r.c[0] & fmask) + (r.dpos & 1u)) * sc;
    const float P1 = small_uint_to_float((r.c[1] & fmask) + ((r.dpos >> 1) & 1u)) * sc;
    const float P2 = small_uint_to_float((r.c[2] & fmask) + ((r.dpos >> 2) & 1u)) * sc;
    // FP32 screen: F_a = fl(fl(P_a ih + nh) + fl(P_a il + nl)) is within 2^-23 |F_a| + 2^-47 (|ih| + |nh|)
    // of the exact crossing time. When the runner-up F_s exceeds the smallest F_b by more than
    // 2^-22 (|F_s| + |F_b|) + 2^-41 max_a (|ih_a| + |nh_a|) (the frame's gscr, over the axes with d_a != 0; the
    // others evaluate to kBigF exactly), F_b's face is the exit face,
    // at least 2^-44 (|ih_b| + |ih_s|) ahead of the others in double-float time: only its double-float
    // time is formed. Otherwise (the ray passes within about 2^-22 frame units of an edge of the leaf) the
    // face is chosen in FP64 from the exact planes.
    float teh, tel, inv_ax;
    int ax;
    bool have64 = false;
    double te64 = 0.0;
    {
        const float F0 = __fadd_rn(__fmaf_rn(P0, r.ih[0], r.nh[0]), __fmaf_rn(P0, r.il[0], r.nl[0]));
        const float F1 = __fadd_rn(__fmaf_rn(P1, r.ih[1], r.nh[1]), __fmaf_rn(P1, r.il[1], r.nl[1]));
        const float F2 = __fadd_rn(__fmaf_rn(P2, r.ih[2], r.nh[2]), __fmaf_rn(P2, r.il[2], r.nl[2]));
        ax = 0;
        float Fb = F0;
        if (F1 < Fb) { ax = 1; Fb = F1; }
        if (F2 < Fb) { ax = 2; Fb = F2; }
        const float Fs = fmaxf(fminf(F0, F1), fminf(fmaxf(F0, F1), F2));  // the median: runner-up
        const bool clear = __fsub_rn(Fs, Fb) > __fmaf_rn(kEps22, __fadd_rn(fabsf(Fs), fabsf(Fb)), r.gscr);
        if (clear) {
            inv_ax = pick(ax, r.ih[0], r.ih[1], r.ih[2]);
            df_cross(pick(ax, P0, P1, P2), inv_ax, pick(ax, r.il[0], r.il[1], r.il[2]), pick(ax, r.nh[0], r.nh[1], r.nh[2]),
                     pick(ax, r.nl[0], r.nl[1], r.nl[2]), teh, tel);
        } else {
            // near an edge: the smallest FP64 crossing time of the exact far planes, ties to the lowest axis
            const Exit64 e = exit_face64(r.k, r.zmask, r.dpos, r.c[0], r.c[1], r.c[2], r.L, T.extent, T.half);
            ax = e.ax;
            inv_ax = pick(ax, r.ih[0], r.ih[1], r.ih[2]);
            te64 = e.t;
            teh = e.hi;
            tel = e.lo;
            have64 = true;
        }
    }
    // 2. neighbour across the exit face
    const uint32_t up = (r.dpos >> ax) & 1u;
    const uint32_t cold = pick(ax, r.c[0], r.c[1], r.c[2]);
    const uint32_t cn = up ? cold + 1u : cold - 1u;
    const int Lold = r.L;
    float base_ax = 0.0f;  // the child-side screen's per-step term (see child_side), with margin 2^-44 |inv_ax|
    auto need64 = [&]() {
        if (!have64) {
            te64 = face_t64(r, T, ax, cold + up, Lold);
            have64 = true;
            split_local(r, te64, teh, tel);
            base_ax = __fmaf_rn(kEps21, fabsf(teh), __fadd_rn(r.gscr, kEpsDF * fabsf(inv_ax)));
            r.k->n_f64 += 1;
        }
        return te64;
    };
    const bool leaves_canvas = (cn >> r.L) != 0u;
    uint32_t cc[3] = {ax == 0 ? cn : r.c[0], ax == 1 ? cn : r.c[1], ax == 2 ? cn : r.c[2]};
    int Lc = r.L, Ln = r.L;
    int32_t prec = 0;
    int kk = 0;
    uint2 nval = make_uint2(0u, 0u);  // the next leaf's value (empty past the canvas)
    bool rebase = false, frame_exit = false;
    if (!leaves_canvas) {
        const int lstar = r.L - (32 - __clz(cold ^ cn));
        const bool fexit = lstar < r.f;
        if (fexit) need64();
        // 3. the new leaf: start at the neighbouring cell (a sibling, the parent's neighbour link,
        //    or the common ancestor on the stack), then descend while the cell is internal
        int lv;  // level of the cell in slot (prec, kk)
        if (kRopes) {
            if (lstar == r.L - 1) {
                prec = r.pr;
                kk = (int)(r.kc ^ (1u << ax));
                lv = r.L;
            } else {
                const uint2 rp = __ldg(T.ropes + (int64_t)r.pr * 6 + 2 * ax + (int)up);
                if (kCount) r.n_rec += 1;
                prec = (int32_t)rp.x;
                kk = (int)((rp.y >> 8) & 7u);
                lv = (int)(rp.y & 255u);
            }
        } else {
            prec = stk[lstar];
            lv = lstar + 1;
            const int sh = Lc - lv;
            kk = (int)((cc[0] >> sh) & 1u) | (int)(((cc[1] >> sh) & 1u) << 1) | (int)(((cc[2] >> sh) & 1u) << 2);
        }
        int32_t slot = load_slot<kSmem>(T, P.smem_records, prec, kk);
        if (kCount) r.n_rec += 1;
        base_ax = __fmaf_rn(kEps21, fabsf(teh), __fadd_rn(r.gscr, kEpsDF * fabsf(inv_ax)));
        while (slot > 0) {
            // internal cell at level lv (record `slot`): choose its child at level lv + 1
            if (!kRopes) stk[lv] = slot;
            int k;
            if (lv < Lc) {
                const int sh = Lc - 1 - lv;
                k = (int)((cc[0] >> sh) & 1u) | (int)(((cc[1] >> sh) & 1u) << 1) | (int)(((cc[2] >> sh) & 1u) << 2);
            } else {
                // finer than the old cell: near side on the exit axis, ray position on the others (FP32
                // screen; FP64 at the exit time for the sides it leaves open, and past a frame exit)
                uint32_t b3[3];
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    b3[a] = a == ax ? (up ? 0u : 1u)
                                    : (fexit ? kUndecided : child_side(r, a, cc[a], lv, teh, tel, base_ax));
                if (b3[0] == kUndecided || b3[1] == kUndecided || b3[2] == kUndecided) {
                    const double t64 = need64();
#pragma unroll
                    for (int a = 0; a < 3; ++a)
                        if (b3[a] == kUndecided) b3[a] = side64(r, T, a, cc[a], lv, t64);
                }
                k = 0;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    cc[a] = 2u * cc[a] + b3[a];
                    k |= (int)b3[a] << a;
                }
                ++Lc;
            }
            prec = slot;
            kk = k;
            ++lv;
            slot = load_slot<kSmem>(T, P.smem_records, prec, kk);
            if (kCount) r.n_rec += 1;
        }
        Ln = lv;
        if (kCount) r.n_reads += (uint32_t)(Ln - lstar);
        if (slot < 0) {
            nval = load_leaf(T, prec, kk, slot);
            if (kCount) r.n_leaf += 1;
        }
        rebase = fexit || (Ln - r.f > P.frame_levels);
        frame_exit = fexit;
    }
    // 4. precision of this boundary (past the canvas: a boundary to sigma = 0)
    if (!have64) {
        if (rebase) {
            need64();
        } else if (nval.x != r.val.x || nval.y != r.val.y) {
            const float need = r.T * fmaxf(hsig(r.val), hsig(nval)) * r.sf_eps * fabsf(inv_ax);
            if (ERR(r) + need > P.err_budget) need64();
            else ERR(r) += need;
        }
    }
    // 5. composite the current leaf, then terminate or advance
    composite(r, teh, tel);
    bool end = leaves_canvas || r.T < P.t_min;
    if (!end && r.steps >= P.step_limit) {
        atomicOr(&P.scratch->status, 1ull);
        atomicAdd(&P.scratch->stats[kStatStepLimited], 1ull);
        end = true;
    }
    if (end) {
        finish(r, P);
        return false;
    }
    const int sh = Lc - Ln;
    r.c[0] = cc[0] >> sh;
    r.c[1] = cc[1] >> sh;
    r.c[2] = cc[2] >> sh;
    r.L = Ln;
    r.val = nval;
    if (kRopes) {
        r.pr = prec;
        r.kc = (uint32_t)kk;
    }
    r.steps += 1;
    if (rebase) {
        // a frame exit takes the coarsest frame that holds the new leaf; a descent past the frame the
        // deepest one the canvas can need, so that deeper leaves do not rebase again level by level
        r.f = frame_exit ? max(0, Ln - P.frame_levels) : deep_frame(Ln, T.depth, P.frame_levels);
        set_frame(r, T, inv_extent, te64);
    } else {
        r.cur_hi = teh;
        r.cur_lo = tel;
    }
    return true;
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    return v;
}

template <bool kSmem, bool kRopes, bool kCount>
__global__ void __launch_bounds__(kBlock, CANVOX_MIN_BLOCKS) mixed_kernel(MixedParams P) {
    __shared__ Cold cold[kBlock];
    __shared__ float2 accs[3 * kBlock];
    __shared__ float errs[kBlock];
    if (kSmem) {
        for (int i = threadIdx.x; i < P.smem_records * 8; i += blockDim.x) s_nodes[i] = __ldg(P.tree.nodes + i);
        __syncthreads();
    }
    int32_t stk[kRopes ? 1 : kMaxDepth + 1];  // ancestors by level (stack traversal only)
    Ray r;
    r.k = &cold[threadIdx.x];
    r.acc = &accs[threadIdx.x];
    r.err = &errs[threadIdx.x];
    r.k->n_rays = r.k->n_steps = r.k->n_f64 = r.k->n_rebase = 0;
    r.n_reads = r.n_leaf = r.n_rec = 0;
    const double inv_extent = 1.0 / P.tree.extent;
    const unsigned lane = threadIdx.x & 31u;
    bool alive = false;
    bool drained = false;
    for (;;) {
        unsigned busy = __ballot_sync(kFull, alive);
        if (!drained && __popc(busy) <= P.refill) {
            const unsigned idle = ~busy;
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(P.queue, (unsigned long long)__popc(idle));
            base = __shfl_sync(kFull, base, 0);
            if (base + __popc(idle) >= (unsigned long long)P.total_rays) drained = true;
            if (!alive) {
                const unsigned long long g = base + __popc(idle & ((1u << lane) - 1u));
                if (g < (unsigned long long)P.total_rays) alive = ray_init<kSmem, kRopes, kCount>(r, P, inv_extent, g, stk);
            }
            busy = __ballot_sync(kFull, alive);
            if (!drained && __popc(busy) <= P.refill) continue;
        }
        if (busy == 0u) {
            if (drained) break;
            continue;
        }
        do {
            if (alive) alive = ray_step<kSmem, kRopes, kCount>(r, P, inv_extent, stk);
            busy = __ballot_sync(kFull, alive);
            // (refill 0, the default: run until every lane is done; the uniform test skips the count)
        } while (busy != 0u && (drained || P.refill == 0 || __popc(busy) > P.refill));
    }
    const unsigned long long v[7] = {r.k->n_rays, r.k->n_steps, kCount ? r.n_reads : 0u, kCount ? r.n_leaf : 0u,
                                     kCount ? r.n_rec : 0u, r.k->n_f64, r.k->n_rebase};
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        const unsigned long long s = warp_sum(v[i]);
        if (lane == 0 && s) atomicAdd(&P.scratch->stats[i], s);
    }
}

}  // namespace

template <bool kRopes, bool kCount>
cudaError_t launch_mixed_t(const MixedParams& p, int grid, int block, cudaStream_t s) {
    if (p.smem_records <= 0) {
        mixed_kernel<false, kRopes, kCount><<<grid, block, 0, s>>>(p);
        return cudaGetLastError();
    }
    // static (per-lane records) plus dynamic shared memory passes the 48 KB default: always opt in
    const int smem = p.smem_records * 32;
    const cudaError_t e =
        cudaFuncSetAttribute(mixed_kernel<true, kRopes, kCount>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    mixed_kernel<true, kRopes, kCount><<<grid, block, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_mixed(const MixedParams& p, int grid, int block, cudaStream_t s) {
    const bool ropes = p.use_ropes && p.tree.ropes;
    if (p.count_reads)
        return ropes ? launch_mixed_t<true, true>(p, grid, block, s) : launch_mixed_t<false, true>(p, grid, block, s);
    return ropes ? launch_mixed_t<true, false>(p, grid, block, s) : launch_mixed_t<false, false>(p, grid, block, s);
}

cudaError_t mixed_max_blocks_per_sm(int block, int smem_bytes, int* out) {
    // all instances share the register and static shared-memory budget
    if (smem_bytes <= 0) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, mixed_kernel<false, true, true>, block, 0);
    cudaError_t e = cudaSuccess;
    const void* fns[4] = {(const void*)mixed_kernel<true, true, true>, (const void*)mixed_kernel<true, false, true>,
                          (const void*)mixed_kernel<true, true, false>, (const void*)mixed_kernel<true, false, false>};
    for (int i = 0; i < 4 && e == cudaSuccess; ++i)
        e = cudaFuncSetAttribute(fns[i], cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, mixed_kernel<true, true, true>, block, smem_bytes);
}

}  // namespace canvox
