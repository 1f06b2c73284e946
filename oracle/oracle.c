/*
 * FP64 CPU oracle for deep-octree ray casting. TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load this library. The product renderer never calls it; it shares no code,
 * header or table with the CUDA path.
 *
 * What it computes (plain definition; Sec. 6 of the paper, with the readings
 * listed in the design notes):
 *   per pixel a ray r(t) = o + t d, |d| = 1, from the eye through the pixel
 *   centre (Sec. 6.1: the eye is kept in FP64 canvas coordinates); the ray is
 *   clipped to the canvas [-E/2, E/2]^3 and to t >= 0. Along it the extinction
 *   sigma and colour c are piecewise constant over the octree leaves. The pixel
 *   is the emission-absorption integral evaluated exactly per leaf segment:
 *       C += T (1 - exp(-sigma l)) c,   T *= exp(-sigma l),
 *   front to back, stopping when T < T_min or at the canvas exit (Sec. 6.2: a
 *   ray ends once it is opaque or leaves the canvas), and
 *   out = (C + T bg.rgb, 1 - T).
 *
 * How: every step locates the leaf that holds the ray just after the current
 * parameter t by descending from the root (no stack, no local frames). On axis
 * a the ray is on the high side of a cell's mid-plane M just after t iff
 *     d_a > 0 : (M - o_a)/d_a <= t,   d_a < 0 : (M - o_a)/d_a > t,
 *     d_a = 0 : o_a >= M.
 * The leaf is left at t_e = min over axes of (far_a - o_a)/d_a (ties: lowest
 * axis). Every plane is an exact dyadic FP64 value; every crossing time uses
 * the same formula, so t increases strictly and each plane is crossed once.
 *
 * Pools (Sec. 4.1.1): record r = 8 int32 slots, child k = x + 2y + 4z;
 * slot > 0 child record, 0 empty leaf, < 0 leaf -slot-1 with FP16 (R,G,B,sigma).
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double eye[3], right[3], up[3], forward[3];
    double tan_half_fov_y;
    int32_t width, height;
    int64_t out_offset_px;
    float background[4];
} ocam;

typedef struct {
    const int32_t *nodes;
    const uint16_t *leaves;
    int32_t depth;
    double extent;
} otree;

/* IEEE 754 binary16 -> double (exact): sign, 5-bit exponent (bias 15), 10-bit fraction. */
static double half_to_double(uint16_t h) {
    int s = h >> 15, e = (h >> 10) & 31, m = h & 1023;
    double v;
    if (e == 0) v = ldexp((double)m, -24);
    else if (e == 31) v = m ? NAN : INFINITY;
    else v = ldexp((double)(m + 1024), e - 25);
    return s ? -v : v;
}

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* Orthonormal camera frame by Gram-Schmidt starting from forward. */
static void camera_frame(const ocam *c, double f[3], double u[3], double r[3]) {
    double n = sqrt(dot3(c->forward, c->forward));
    for (int a = 0; a < 3; ++a) f[a] = c->forward[a] / n;
    double uf = dot3(c->up, f);
    for (int a = 0; a < 3; ++a) u[a] = c->up[a] - uf * f[a];
    n = sqrt(dot3(u, u));
    for (int a = 0; a < 3; ++a) u[a] /= n;
    double rf = dot3(c->right, f), ru = dot3(c->right, u);
    for (int a = 0; a < 3; ++a) r[a] = c->right[a] - rf * f[a] - ru * u[a];
    n = sqrt(dot3(r, r));
    for (int a = 0; a < 3; ++a) r[a] /= n;
}

/* Unit direction through the centre of pixel (i, j); j counts rows from the top. */
static void pixel_ray(const ocam *c, const double f[3], const double u[3], const double r[3],
                      int64_t i, int64_t j, double d[3]) {
    double aspect = (double)c->width / (double)c->height;
    double px = (2.0 * ((double)i + 0.5) / (double)c->width - 1.0) * c->tan_half_fov_y * aspect;
    double py = (1.0 - 2.0 * ((double)j + 0.5) / (double)c->height) * c->tan_half_fov_y;
    for (int a = 0; a < 3; ++a) d[a] = f[a] + px * r[a] + py * u[a];
    double n = sqrt(dot3(d, d));
    for (int a = 0; a < 3; ++a) d[a] /= n;
}

/* Is the ray on the high side of plane x_a = M just after parameter t? */
static int high_side(double M, double o, double d, double t) {
    if (d > 0.0) return (M - o) / d <= t;
    if (d < 0.0) return (M - o) / d > t;
    return o >= M;
}

typedef struct {
    int64_t steps, reads, leaf_loads;
    double sum_width, length;
    int guard;
} ocount;

/* Render one ray; writes rgba[4] and the counters. */
static void trace(const otree *T, const double o[3], const double d[3], const float bg[4],
                  double t_min, int64_t max_steps, double rgba[4], ocount *cnt,
                  unsigned char *rec_mark, unsigned char *leaf_mark) {
    const double E = T->extent, h = 0.5 * E;
    memset(cnt, 0, sizeof(*cnt));
    /* clip to the canvas: inside on axis a just after t iff enter_a <= t < exit_a */
    double t0 = 0.0, t1 = INFINITY;
    for (int a = 0; a < 3; ++a) {
        if (d[a] > 0.0) {
            double te = (-h - o[a]) / d[a], tx = (h - o[a]) / d[a];
            if (te > t0) t0 = te;
            if (tx < t1) t1 = tx;
        } else if (d[a] < 0.0) {
            double te = (h - o[a]) / d[a], tx = (-h - o[a]) / d[a];
            if (te > t0) t0 = te;
            if (tx < t1) t1 = tx;
        } else if (!(o[a] >= -h && o[a] < h)) {
            t1 = -INFINITY;
        }
    }
    double C[3] = {0.0, 0.0, 0.0}, Tr = 1.0;
    if (t0 < t1) {
        int prev_path[32];
        int prev_len = -1;
        double t = t0;
        for (;;) {
            if (cnt->steps >= max_steps) { cnt->guard = 1; break; }
            /* locate the leaf holding r(t+) from the root */
            double lo[3] = {-h, -h, -h}, w = E;
            int32_t rec = 0, slot = 0;
            int path[32], L = 0;
            for (;;) {
                double hw = 0.5 * w;
                int k = 0;
                for (int a = 0; a < 3; ++a) {
                    double M = lo[a] + hw;
                    if (high_side(M, o[a], d[a], t)) { k |= 1 << a; lo[a] = M; }
                }
                w = hw;
                path[L++] = k;
                if (rec_mark) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
                    rec_mark[rec] = 1;
                }
                slot = T->nodes[8 * (int64_t)rec + k];
                if (slot <= 0) break;
                rec = slot;
            }
            /* LCA with the previous leaf: common prefix of the child paths */
            int common = 0;
            if (prev_len >= 0)
                while (common < L && common < prev_len && path[common] == prev_path[common]) ++common;
            cnt->reads += L - common;
            memcpy(prev_path, path, sizeof(int) * (size_t)L);
            prev_len = L;
            cnt->steps += 1;
            cnt->sum_width += w;
            /* leave the leaf at the nearest far face */
            double te = INFINITY;
            for (int a = 0; a < 3; ++a) {
                if (d[a] == 0.0) continue;
                double far = d[a] > 0.0 ? lo[a] + w : lo[a];
                double ta = (far - o[a]) / d[a];
                if (ta < te) te = ta;
            }
            if (te > t1) te = t1;
            double l = te - t;
            if (slot < 0) {
                const uint16_t *v = T->leaves + 4 * (int64_t)(-slot - 1);
                double sg = half_to_double(v[3]);
                cnt->leaf_loads += 1;
                if (leaf_mark) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
                    leaf_mark[-slot - 1] = 1;
                }
                if (sg > 0.0) {
                    double a = -expm1(-sg * l);
                    for (int c = 0; c < 3; ++c) C[c] += Tr * a * half_to_double(v[c]);
                    Tr *= exp(-sg * l);
                }
            }
            if (Tr < t_min || te >= t1) { cnt->length = te - t0; break; }
            t = te;
        }
    }
    for (int c = 0; c < 3; ++c) rgba[c] = C[c] + Tr * (double)bg[c];
    rgba[3] = 1.0 - Tr;
}

/*
 * oracle_render: render the listed output pixels (or, when px_idx is NULL, every pixel of
 * every view, indexed by output pixel). out_rgba: n x 4 doubles. Optional
 * counters: icount n x 3 (steps, slot reads from the LCA, leaf loads) and
 * dcount n x 2 (sum of crossed cell widths, ray length in the canvas).
 * Returns 0, -1 for bad arguments, or the number of rays that hit the
 * step guard (an oracle bug; those pixels are NaN).
 */
static int64_t render_pixels(const int32_t *nodes, const uint16_t *leaves, int32_t depth, double extent,
                             const ocam *cams, int32_t n_views, const int64_t *px_idx, int64_t n_px,
                             double t_min, int64_t max_steps, double *out_rgba, int64_t *icount, double *dcount,
                             int32_t n_threads, unsigned char *rec_mark, unsigned char *leaf_mark) {
    if (!nodes || depth < 1 || depth > 30 || !(extent > 0.0) || n_views < 0 || (n_views && !cams) || !out_rgba)
        return -1;
    otree T = {nodes, leaves, depth, extent};
    if (max_steps <= 0) max_steps = 3 * ((int64_t)1 << depth) + 8;
    int64_t total = 0;
    for (int v = 0; v < n_views; ++v) {
        int64_t e = cams[v].out_offset_px + (int64_t)cams[v].width * cams[v].height;
        if (e > total) total = e;
    }
    int64_t n = px_idx ? n_px : total;
    int64_t bad = 0;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : bad)
#endif
    for (int64_t q = 0; q < n; ++q) {
        int64_t p = px_idx ? px_idx[q] : q;
        double *out = out_rgba + 4 * q;
        int found = -1;
        for (int v = 0; v < n_views; ++v) {
            int64_t np = (int64_t)cams[v].width * cams[v].height;
            if (p >= cams[v].out_offset_px && p < cams[v].out_offset_px + np) { found = v; break; }
        }
        ocount cnt;
        memset(&cnt, 0, sizeof(cnt));
        if (found < 0) {
            out[0] = out[1] = out[2] = out[3] = NAN;
        } else {
            const ocam *c = &cams[found];
            int64_t local = p - c->out_offset_px;
            double f[3], u[3], r[3], d[3];
            camera_frame(c, f, u, r);
            pixel_ray(c, f, u, r, local % c->width, local / c->width, d);
            trace(&T, c->eye, d, c->background, t_min, max_steps, out, &cnt, rec_mark, leaf_mark);
            if (cnt.guard) { out[0] = out[1] = out[2] = out[3] = NAN; bad += 1; }
        }
        if (icount) { icount[3 * q] = cnt.steps; icount[3 * q + 1] = cnt.reads; icount[3 * q + 2] = cnt.leaf_loads; }
        if (dcount) { dcount[2 * q] = cnt.sum_width; dcount[2 * q + 1] = cnt.length; }
    }
    return bad;
}

int64_t oracle_render(const int32_t *nodes, const uint16_t *leaves, int32_t depth, double extent,
                      const ocam *cams, int32_t n_views, const int64_t *px_idx, int64_t n_px,
                      double t_min, int64_t max_steps, double *out_rgba, int64_t *icount, double *dcount,
                      int32_t n_threads) {
    return render_pixels(nodes, leaves, depth, extent, cams, n_views, px_idx, n_px, t_min, max_steps, out_rgba,
                         icount, dcount, n_threads, NULL, NULL);
}

/*
 * Render every pixel (out_rgba: one row of 4 doubles per output pixel) and
 * mark the records this traversal reads (every record on the root-to-leaf path
 * of every step) and the stored leaves it loads: rec_mark[n_records] and
 * leaf_mark[n_leaves] bytes, set to 1. This is the footprint of the traversal
 * (the distinct data a render from a cold cache must read).
 */
int64_t oracle_footprint(const int32_t *nodes, const uint16_t *leaves, int32_t depth, double extent,
                         const ocam *cams, int32_t n_views, double t_min, double *out_rgba,
                         unsigned char *rec_mark, unsigned char *leaf_mark, int32_t n_threads) {
    if (!rec_mark || !leaf_mark) return -1;
    return render_pixels(nodes, leaves, depth, extent, cams, n_views, NULL, 0, t_min, 0, out_rgba, NULL, NULL,
                         n_threads, rec_mark, leaf_mark);
}

/* Trace explicit rays (origin, direction not necessarily unit). For tests of single rays. */
int64_t oracle_trace_rays(const int32_t *nodes, const uint16_t *leaves, int32_t depth, double extent,
                          const double *orig, const double *dir, int64_t n, const float *bg, double t_min,
                          int64_t max_steps, double *out_rgba, int64_t *icount, double *dcount) {
    if (!nodes || depth < 1 || depth > 30 || !(extent > 0.0)) return -1;
    otree T = {nodes, leaves, depth, extent};
    if (max_steps <= 0) max_steps = 3 * ((int64_t)1 << depth) + 8;
    int64_t bad = 0;
    for (int64_t q = 0; q < n; ++q) {
        double d[3] = {dir[3 * q], dir[3 * q + 1], dir[3 * q + 2]};
        double nn = sqrt(dot3(d, d));
        for (int a = 0; a < 3; ++a) d[a] /= nn;
        ocount cnt;
        trace(&T, orig + 3 * q, d, bg, t_min, max_steps, out_rgba + 4 * q, &cnt, NULL, NULL);
        if (cnt.guard) bad += 1;
        if (icount) { icount[3 * q] = cnt.steps; icount[3 * q + 1] = cnt.reads; icount[3 * q + 2] = cnt.leaf_loads; }
        if (dcount) { dcount[2 * q] = cnt.sum_width; dcount[2 * q + 1] = cnt.length; }
    }
    return bad;
}

/* Number of OpenMP threads a parallel region would use (1 without OpenMP). */
int32_t oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
