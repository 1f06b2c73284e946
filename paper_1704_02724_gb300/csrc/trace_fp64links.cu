// FP64 twin of the mixed-precision traversal: the precision comparator.
//
// The same traversal as the mixed kernel (trace_mixed.cu): a persistent grid
// whose warps pop tiles of rays from one global queue, exact integer cell
// coordinates, the neighbour found as a sibling or through the parent's
// neighbour link (the neighbour graph of Sec. 4.1.1, built at upload), a
// descent while the cell is internal, front-to-back compositing to full
// opacity or the canvas exit (Sec. 6.2). What differs is the arithmetic:
// every crossing time is FP64 from the exact plane, t = P inv + nod in canvas
// coordinates (no local frame, no FP32 screen, no error budget), every side
// test is FP64, and colour and transmittance are FP64 sums. Timing this kernel
// beside the mixed one isolates what the local frames of Sec. 6.1-6.3 buy on
// this GPU, whose FP64 rate is a small fraction of its FP32 rate; the plain FP64
// caster (trace_plain.cu) differs from the mixed kernel in its traversal too.
//
// Decisions follow the FP64 oracle's conventions: a ray leaves a leaf by the
// face with the smallest crossing time (ties to the lowest axis), and is on the
// high side of a plane M just after t iff (M - o)/d <= t for d > 0, > t for
// d < 0, and o >= M for d = 0 (here with the product form M inv + nod).
#include <cuda_fp16.h>

#include "canvox_internal.cuh"

namespace canvox {
namespace {

constexpr unsigned kFull64 = 0xFFFFFFFFu;
constexpr int kBlock64 = 256;

__device__ __forceinline__ double p2d(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }
__device__ __forceinline__ double h2d(unsigned h) { return (double)__half2float(__ushort_as_half((unsigned short)h)); }

// FP64 state of a lane that the step reads rarely: the output address and the colour sums.
struct Cold64 {
    double C[3];
    uint32_t pix;
    int32_t view;
};

struct Ray64 {
    Cold64* k;
    double inv[3], nod[3];  // t(X) = X inv + nod; axis with d = 0: inv = 0, nod = o
    double t;               // parameter where the current leaf is entered
    double T;               // transmittance
    uint32_t c[3];
    int32_t L;
    uint32_t dpos, zmask;
    uint2 val;
    int32_t pr;   // record holding the current leaf's slot
    uint32_t kc;  // child index of the current leaf in pr
    int32_t steps;
    uint32_t n_rays, n_steps, n_reads, n_leaf, n_rec;
};

__device__ __forceinline__ bool zero_axis(const Ray64& r, int a) { return (r.zmask >> a) & 1u; }

// Ray on the high side of the plane x_a = M just after t.
__device__ __forceinline__ uint32_t high_side(const Ray64& r, int a, double M, double t) {
    if (zero_axis(r, a)) return r.nod[a] >= M;
    const double tm = fma(M, r.inv[a], r.nod[a]);
    return r.inv[a] > 0.0 ? (tm <= t) : (tm > t);
}

__device__ __forceinline__ double mid_plane(const Tree& T, uint32_t cc, int lev) {
    return fma((double)(2u * cc + 1u), T.extent * p2d(-(lev + 1)), -T.half);
}

// Composite the current leaf over [r.t, te].
__device__ __forceinline__ void composite64(Ray64& r, double te) {
    if (r.val.y >> 16) {
        const double s = h2d(r.val.y >> 16);
        const double em = expm1(-s * (te - r.t));  // -(1 - e^{-sigma l})
        const double w = -r.T * em;
        r.k->C[0] += w * h2d(r.val.x & 0xFFFFu);
        r.k->C[1] += w * h2d(r.val.x >> 16);
        r.k->C[2] += w * h2d(r.val.y & 0xFFFFu);
        r.T += r.T * em;
    }
}

__device__ __forceinline__ void finish64(Ray64& r, const MixedParams& P) {
    const View& V = P.views[r.k->view];
    float4 o;
    o.x = (float)(r.k->C[0] + r.T * (double)V.bg[0]);
    o.y = (float)(r.k->C[1] + r.T * (double)V.bg[1]);
    o.z = (float)(r.k->C[2] + r.T * (double)V.bg[2]);
    o.w = (float)(1.0 - r.T);
    const int64_t pix = V.out_offset + (int64_t)r.k->pix;
    P.out[pix] = o;
    if (P.step_count) P.step_count[pix] = r.steps;
    r.n_rays += 1;
    r.n_steps += (uint32_t)r.steps;
}

// Start ray g of the launch. Returns true if it has a leaf to step from.
__device__ bool init64(Ray64& r, const MixedParams& P, unsigned long long g) {
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
    const unsigned tile = (unsigned)(local >> 5);
    const int lane = (int)(local & 31);
    const unsigned ty = tile / (unsigned)V.tiles_x;
    const int wl = V.tile_wl;
    const int i = ((int)(tile - ty * (unsigned)V.tiles_x) << wl) + (lane & ((1 << wl) - 1));
    const int j = (int)ty * (32 >> wl) + (lane >> wl);
    if (i >= V.width || j >= V.height) return false;
    r.k->view = lo;
    r.k->pix = (uint32_t)j * (uint32_t)V.width + (uint32_t)i;
    r.k->C[0] = r.k->C[1] = r.k->C[2] = 0.0;
    r.T = 1.0;
    r.steps = 0;
    double d[3];
    pixel_ray(V, i, j, d);
    r.dpos = 0;
    r.zmask = 0;
    double t0 = 0.0, t1 = __longlong_as_double(0x7FF0000000000000ll);
    bool miss = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double da = d[a], o = V.eye[a];
        if (da != 0.0) {
            r.inv[a] = 1.0 / da;
            r.nod[a] = -o * r.inv[a];
            if (da > 0.0) r.dpos |= 1u << a;
            const double ta = fma(-T.half, r.inv[a], r.nod[a]);
            const double tb = fma(T.half, r.inv[a], r.nod[a]);
            t0 = fmax(t0, da > 0.0 ? ta : tb);
            t1 = fmin(t1, da > 0.0 ? tb : ta);
        } else {
            r.inv[a] = 0.0;
            r.nod[a] = o;
            r.zmask |= 1u << a;
            if (!(o >= -T.half && o < T.half)) miss = true;
        }
    }
    if (miss || !(t0 < t1)) {
        finish64(r, P);
        return false;
    }
    r.t = t0;
    const EyePath& E = P.eye[r.k->view];
    if (E.len > 0 && t0 == 0.0) {
        r.L = E.len;
        r.pr = E.rec[E.len - 1];
        r.kc = (E.c[0] & 1u) | ((E.c[1] & 1u) << 1) | ((E.c[2] & 1u) << 2);
        r.c[0] = E.c[0];
        r.c[1] = E.c[1];
        r.c[2] = E.c[2];
        r.val = E.val;
        r.n_reads += r.L;
        r.n_leaf += (uint32_t)E.stored;
        r.steps = 1;
        return true;
    }
    // locate the leaf that holds r(t0+) from the root
    r.c[0] = r.c[1] = r.c[2] = 0u;
    int lev = 0;
    int32_t rec = 0, slot;
    for (;;) {
        int k = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const uint32_t b = high_side(r, a, mid_plane(T, r.c[a], lev), t0);
            r.c[a] = 2u * r.c[a] + b;
            k |= (int)b << a;
        }
        slot = __ldg(T.nodes + (int64_t)rec * 8 + k);
        r.n_rec += 1;
        if (slot > 0) {
            ++lev;
            rec = slot;
        } else {
            r.pr = rec;
            r.kc = (uint32_t)k;
            break;
        }
    }
    r.L = lev + 1;
    r.n_reads += r.L;
    if (slot < 0) {
        r.val = __ldg(T.leaves + leaf_index(T, rec, (int)r.kc, slot));
        r.n_leaf += 1;
    } else {
        r.val = make_uint2(0u, 0u);
    }
    r.steps = 1;
    return true;
}

// One leaf step. Returns false once the ray is finished (its pixel written).
__device__ bool step64(Ray64& r, const MixedParams& P) {
    const Tree& T = P.tree;
    // 1. exit face: the smallest FP64 crossing time of the exact far planes (ties to the lowest axis)
    const double w = T.extent * p2d(-r.L);
    double te = __longlong_as_double(0x7FF0000000000000ll);
    int ax = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (zero_axis(r, a)) continue;
        const double ta = fma(fma((double)(r.c[a] + ((r.dpos >> a) & 1u)), w, -T.half), r.inv[a], r.nod[a]);
        if (ta < te) {
            te = ta;
            ax = a;
        }
    }
    // 2. neighbour across the exit face
    const uint32_t up = (r.dpos >> ax) & 1u;
    const uint32_t cold = ax == 0 ? r.c[0] : (ax == 1 ? r.c[1] : r.c[2]);
    const uint32_t cn = up ? cold + 1u : cold - 1u;
    if ((cn >> r.L) != 0u) {  // leaving the canvas
        composite64(r, te);
        finish64(r, P);
        return false;
    }
    const int lstar = r.L - (32 - __clz(cold ^ cn));
    uint32_t cc[3] = {ax == 0 ? cn : r.c[0], ax == 1 ? cn : r.c[1], ax == 2 ? cn : r.c[2]};
    int Lc = r.L;
    int lv;
    int32_t prec;
    int kk;
    if (lstar == r.L - 1) {
        prec = r.pr;
        kk = (int)(r.kc ^ (1u << ax));
        lv = r.L;
    } else {
        const uint2 rp = __ldg(T.ropes + (int64_t)r.pr * 6 + 2 * ax + (int)up);
        r.n_rec += 1;
        prec = (int32_t)rp.x;
        kk = (int)((rp.y >> 8) & 7u);
        lv = (int)(rp.y & 255u);
    }
    int32_t slot = __ldg(T.nodes + (int64_t)prec * 8 + kk);
    r.n_rec += 1;
    // 3. descend while the cell is internal: integer bits down to the old level, then the ray's side at te
    while (slot > 0) {
        int k;
        if (lv < Lc) {
            const int sh = Lc - 1 - lv;
            k = (int)((cc[0] >> sh) & 1u) | (int)(((cc[1] >> sh) & 1u) << 1) | (int)(((cc[2] >> sh) & 1u) << 2);
        } else {
            k = 0;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const uint32_t bit = a == ax ? (up ? 0u : 1u) : high_side(r, a, mid_plane(T, cc[a], lv), te);
                cc[a] = 2u * cc[a] + bit;
                k |= (int)bit << a;
            }
            ++Lc;
        }
        prec = slot;
        kk = k;
        ++lv;
        slot = __ldg(T.nodes + (int64_t)prec * 8 + kk);
        r.n_rec += 1;
    }
    const int Ln = lv;
    r.n_reads += (uint32_t)(Ln - lstar);
    uint2 nval = make_uint2(0u, 0u);
    if (slot < 0) {
        nval = __ldg(T.leaves + leaf_index(T, prec, kk, slot));
        r.n_leaf += 1;
    }
    // 4. composite the current leaf, then terminate or advance
    composite64(r, te);
    if (r.T < (double)P.t_min) {
        finish64(r, P);
        return false;
    }
    if (r.steps >= P.step_limit) {
        atomicOr(&P.scratch->status, 1ull);
        atomicAdd(&P.scratch->stats[kStatStepLimited], 1ull);
        finish64(r, P);
        return false;
    }
    const int sh = Lc - Ln;
    r.c[0] = cc[0] >> sh;
    r.c[1] = cc[1] >> sh;
    r.c[2] = cc[2] >> sh;
    r.L = Ln;
    r.val = nval;
    r.pr = prec;
    r.kc = (uint32_t)kk;
    r.t = te;
    r.steps += 1;
    return true;
}

__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull64, v, o);
    return v;
}

__global__ void __launch_bounds__(kBlock64, 3) fp64links_kernel(MixedParams P) {
    __shared__ Cold64 cold[kBlock64];
    Ray64 r;
    r.k = &cold[threadIdx.x];
    r.n_rays = r.n_steps = r.n_reads = r.n_leaf = r.n_rec = 0;
    const unsigned lane = threadIdx.x & 31u;
    bool alive = false;
    bool drained = false;
    for (;;) {
        unsigned busy = __ballot_sync(kFull64, alive);
        if (!drained && __popc(busy) <= P.refill) {
            const unsigned idle = ~busy;
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(P.queue, (unsigned long long)__popc(idle));
            base = __shfl_sync(kFull64, base, 0);
            if (base + __popc(idle) >= (unsigned long long)P.total_rays) drained = true;
            if (!alive) {
                const unsigned long long g = base + __popc(idle & ((1u << lane) - 1u));
                if (g < (unsigned long long)P.total_rays) alive = init64(r, P, g);
            }
            busy = __ballot_sync(kFull64, alive);
            if (!drained && __popc(busy) <= P.refill) continue;
        }
        if (busy == 0u) {
            if (drained) break;
            continue;
        }
        do {
            if (alive) alive = step64(r, P);
            busy = __ballot_sync(kFull64, alive);
        } while (busy != 0u && (drained || __popc(busy) > P.refill));
    }
    const unsigned long long v[5] = {r.n_rays, r.n_steps, r.n_reads, r.n_leaf, r.n_rec};
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const unsigned long long s = warp_sum64(v[i]);
        if (lane == 0 && s) atomicAdd(&P.scratch->stats[i], s);
    }
}

}  // namespace

cudaError_t launch_fp64links(const MixedParams& p, int grid, int block, cudaStream_t s) {
    if (!p.tree.ropes) return cudaErrorInvalidValue;
    fp64links_kernel<<<grid, block, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t fp64links_max_blocks_per_sm(int block, int* out) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, fp64links_kernel, block, 0);
}

}  // namespace canvox
