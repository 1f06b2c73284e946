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
 * slot > 0 child record, 0 empty leaf, < 0 a stored leaf with FP16 (R,G,B,sigma).
 * Stored leaves are numbered 0, 1, ... in breadth-first slot order (records in
 * order, slots k = 0..7 within a record). The oracle takes a leaf's number as
 * that count itself: the leaf slots of the records before it (leaf_base[r],
 * from oracle_leaf_base) plus those before it in its record. It does not read
 * the number the slot stores (the same number, modulo 2^31).
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
    const int64_t *leaf_base;  /* leaf slots in records 0 .. r-1 */
    int32_t depth;
    double extent;
} otree;

/* leaf_base[r] = number of leaf slots (slot < 0) in records 0 .. r-1. */
void oracle_leaf_base(const int32_t *nodes, int64_t n_rec, int64_t *leaf_base) {
    int64_t c = 0;
    for (int64_t r = 0; r < n_rec; ++r) {
        leaf_base[r] = c;
        for (int k = 0; k < 8; ++k) c += nodes[8 * r + k] < 0;
    }
}

/* Number of the stored leaf in slot k of record rec: the leaf slots before it in breadth-first slot order. */
static int64_t leaf_number(const otree *T, int32_t rec, int k) {
    int64_t li = T->leaf_base[rec];
    for (int j = 0; j < k; ++j) li += T->nodes[8 * (int64_t)rec + j] < 0;
    return li;
}

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
                const int64_t li = leaf_number(T, rec, path[L - 1]);
                const uint16_t *v = T->leaves + 4 * li;
                double sg = half_to_double(v[3]);
                cnt->leaf_loads += 1;
                if (leaf_mark) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
                    leaf_mark[li] = 1;
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
static int64_t render_pixels(const int32_t *nodes, const uint16_t *leaves, const int64_t *leaf_base, int32_t depth,
                             double extent, const ocam *cams, int32_t n_views, const int64_t *px_idx, int64_t n_px,
                             double t_min, int64_t max_steps, double *out_rgba, int64_t *icount, double *dcount,
                             int32_t n_threads, unsigned char *rec_mark, unsigned char *leaf_mark) {
    if (!nodes || !leaf_base || depth < 1 || depth > 30 || !(extent > 0.0) || n_views < 0 || (n_views && !cams) ||
        !out_rgba)
        return -1;
    otree T = {nodes, leaves, leaf_base, depth, extent};
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

int64_t oracle_render(const int32_t *nodes, const uint16_t *leaves, const int64_t *leaf_base, int32_t depth,
                      double extent, const ocam *cams, int32_t n_views, const int64_t *px_idx, int64_t n_px,
                      double t_min, int64_t max_steps, double *out_rgba, int64_t *icount, double *dcount,
                      int32_t n_threads) {
    return render_pixels(nodes, leaves, leaf_base, depth, extent, cams, n_views, px_idx, n_px, t_min, max_steps,
                         out_rgba, icount, dcount, n_threads, NULL, NULL);
}

/*
 * Render every pixel (out_rgba: one row of 4 doubles per output pixel) and
 * mark the records this traversal reads (every record on the root-to-leaf path
 * of every step) and the stored leaves it loads: rec_mark[n_records] and
 * leaf_mark[n_leaves] bytes, set to 1. This is the footprint of the traversal
 * (the distinct data a render from a cold cache must read).
 */
int64_t oracle_footprint(const int32_t *nodes, const uint16_t *leaves, const int64_t *leaf_base, int32_t depth,
                         double extent, const ocam *cams, int32_t n_views, double t_min, double *out_rgba,
                         unsigned char *rec_mark, unsigned char *leaf_mark, int32_t n_threads) {
    if (!rec_mark || !leaf_mark) return -1;
    return render_pixels(nodes, leaves, leaf_base, depth, extent, cams, n_views, NULL, 0, t_min, 0, out_rgba, NULL,
                         NULL, n_threads, rec_mark, leaf_mark);
}

/* Trace explicit rays (origin, direction not necessarily unit). For tests of single rays. */
int64_t oracle_trace_rays(const int32_t *nodes, const uint16_t *leaves, const int64_t *leaf_base, int32_t depth,
                          double extent, const double *orig, const double *dir, int64_t n, const float *bg,
                          double t_min, int64_t max_steps, double *out_rgba, int64_t *icount, double *dcount) {
    if (!nodes || !leaf_base || depth < 1 || depth > 30 || !(extent > 0.0)) return -1;
    otree T = {nodes, leaves, leaf_base, depth, extent};
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

/*
 * The paper's single-precision walks (Sec. 6.2-6.3), geometry only, as the check of the
 * GPU's implementation of them: the ray's position is carried in FP32, either in the
 * frame of the current cell (cell_local = 1: origin at the cell centre, unit size,
 * p in [-0.5, 0.5]) or in canvas coordinates (cell_local = 0). Each step leaves the
 * cell at the nearest face, t = (face - p_a)/d_a, moves to p' = p + t d (the exit
 * coordinate set to the face in the cell frame), finds the neighbour from integer
 * cell coordinates, and re-expresses p' in the neighbour's frame: one cell over on
 * the exit axis; for a finer neighbour, halving into the child the point lies in
 * (2q -+ 1/2); for a coarser one, p' s + c with s the ratio of cell sizes and c the
 * offset of the centres. Every FP32 operation is rounded on its own (no contraction).
 * The start point is the canvas entry in FP64 (fma(t0, d, o)) rounded into the frame,
 * and the start leaf is located in FP64 as in the ray caster above. The walk runs to
 * the canvas exit (no compositing), and per output pixel writes the leaves visited
 * and the angle in degrees between the pixel direction d and the line from the eye
 * to the final position, atan2(|v x d|, v . d), v = X - o. Pixels of no view: -1, NaN.
 */
static float rel_face(float p, float d) { return (d > 0.0f ? 0.5f : -0.5f) - p; }

int64_t oracle_walk32(const int32_t *nodes, int32_t depth, double extent, const ocam *cams, int32_t n_views,
                      int32_t cell_local, int64_t max_steps, int32_t *steps_out, double *angle_out,
                      int32_t n_threads) {
    if (!nodes || depth < 1 || depth > 30 || !(extent > 0.0) || n_views < 0 || (n_views && !cams)) return -1;
    if (max_steps <= 0) max_steps = 3 * ((int64_t)1 << depth) + 8;
    const double E = extent, h = 0.5 * extent;
    int64_t total = 0;
    for (int v = 0; v < n_views; ++v) {
        int64_t e = cams[v].out_offset_px + (int64_t)cams[v].width * cams[v].height;
        if (e > total) total = e;
    }
    for (int64_t q = 0; q < total; ++q) {
        steps_out[q] = -1;
        angle_out[q] = NAN;
    }
    int64_t bad = 0;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#endif
    for (int v = 0; v < n_views; ++v) {
        const ocam *cm = &cams[v];
        double f[3], u[3], r[3];
        camera_frame(cm, f, u, r);
        const int64_t npx = (int64_t)cm->width * cm->height;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : bad)
#endif
        for (int64_t local = 0; local < npx; ++local) {
            double d64[3];
            pixel_ray(cm, f, u, r, local % cm->width, local / cm->width, d64);
            const double *o = cm->eye;
            double t0 = 0.0, t1 = INFINITY;
            int miss = 0;
            for (int a = 0; a < 3; ++a) {
                if (d64[a] != 0.0) {
                    double ta = (-h - o[a]) / d64[a], tb = (h - o[a]) / d64[a];
                    t0 = fmax(t0, d64[a] > 0.0 ? ta : tb);
                    t1 = fmin(t1, d64[a] > 0.0 ? tb : ta);
                } else if (!(o[a] >= -h && o[a] < h)) {
                    miss = 1;
                }
            }
            int32_t steps = 0;
            double angle = 0.0;
            if (!miss && t0 < t1) {
                /* start leaf holding r(t0+) */
                uint32_t c[3] = {0, 0, 0};
                int L = 0;
                int32_t rec = 0, slot;
                for (;;) {
                    double w = ldexp(E, -(L + 1));
                    int k = 0;
                    for (int a = 0; a < 3; ++a) {
                        double M = fma((double)(2u * c[a] + 1u), w, -h);
                        uint32_t b = (uint32_t)high_side(M, o[a], d64[a], t0);
                        c[a] = 2u * c[a] + b;
                        k |= (int)b << a;
                    }
                    slot = nodes[8 * (int64_t)rec + k];
                    ++L;
                    if (slot <= 0) break;
                    rec = slot;
                }
                const float d[3] = {(float)d64[0], (float)d64[1], (float)d64[2]};
                float p[3];
                double X[3];
                for (int a = 0; a < 3; ++a) {
                    double x = fma(t0, d64[a], o[a]);
                    X[a] = x;
                    if (cell_local) {
                        double w = ldexp(E, -L);
                        double centre = fma((double)c[a] + 0.5, w, -h);
                        p[a] = (float)((x - centre) / w);
                    } else {
                        p[a] = (float)x;
                    }
                }
                for (;;) {
                    if (steps >= max_steps) { bad += 1; break; }
                    steps += 1;
                    const double w64 = ldexp(E, -L);
                    float te = INFINITY;
                    int ax = -1;
                    for (int a = 0; a < 3; ++a) {
                        if (d[a] == 0.0f) continue;
                        float num = cell_local ? rel_face(p[a], d[a])
                                               : (float)fma((double)(c[a] + (d[a] > 0.0f ? 1u : 0u)), w64, -h) - p[a];
                        float ta = num / d[a];
                        if (ta < te) { te = ta; ax = a; }
                    }
                    if (ax < 0) break;
                    float pe[3];
                    for (int a = 0; a < 3; ++a) {
                        float m = te * d[a];
                        pe[a] = p[a] + m;
                    }
                    if (cell_local) pe[ax] = d[ax] > 0.0f ? 0.5f : -0.5f;
                    for (int a = 0; a < 3; ++a)
                        X[a] = cell_local ? fma((double)c[a] + 0.5 + (double)pe[a], w64, -h) : (double)pe[a];
                    const uint32_t up = d[ax] > 0.0f ? 1u : 0u;
                    const uint32_t cn = up ? c[ax] + 1u : c[ax] - 1u;
                    if ((cn >> L) != 0u) break;
                    /* the neighbour: from the root by integer coordinates, at most level L */
                    uint32_t cc[3] = {c[0], c[1], c[2]};
                    cc[ax] = cn;
                    int Ln = 0;
                    rec = 0;
                    for (int lev = 0;; ++lev) {
                        int sh = L - 1 - lev, k = 0;
                        for (int a = 0; a < 3; ++a) k |= (int)((cc[a] >> sh) & 1u) << a;
                        slot = nodes[8 * (int64_t)rec + k];
                        if (slot <= 0 || lev + 1 == L) { Ln = lev + 1; break; }
                        rec = slot;
                    }
                    float qv[3] = {pe[0], pe[1], pe[2]};
                    if (cell_local) qv[ax] = up ? -0.5f : 0.5f;
                    int Lc = L;
                    while (slot > 0) {
                        /* finer neighbour: near side on the exit axis, the FP32 position on the others */
                        rec = slot;
                        int k = 0;
                        double wc = ldexp(E, -(Lc + 1));
                        for (int a = 0; a < 3; ++a) {
                            uint32_t b;
                            if (a == ax) {
                                b = up ? 0u : 1u;
                            } else if (cell_local) {
                                b = qv[a] > 0.0f || (qv[a] == 0.0f && d[a] >= 0.0f);
                            } else {
                                float M = (float)fma((double)(2u * cc[a] + 1u), wc, -h);
                                b = qv[a] > M || (qv[a] == M && d[a] >= 0.0f);
                            }
                            if (cell_local) {
                                float twice = 2.0f * qv[a];
                                qv[a] = twice - (b ? 0.5f : -0.5f);
                            }
                            cc[a] = 2u * cc[a] + b;
                            k |= (int)b << a;
                        }
                        ++Lc;
                        slot = nodes[8 * (int64_t)rec + k];
                        Ln = Lc;
                    }
                    if (cell_local && Ln < L) {
                        double s64 = ldexp(1.0, Ln - L);
                        float sf = (float)s64;
                        for (int a = 0; a < 3; ++a) {
                            uint32_t cp = cc[a] >> (L - Ln);
                            double off = ((double)cc[a] + 0.5) * s64 - ((double)cp + 0.5);
                            float scaled = qv[a] * sf;
                            qv[a] = scaled + (float)off;
                        }
                        qv[ax] = up ? -0.5f : 0.5f;
                    }
                    int shn = Lc - Ln;
                    for (int a = 0; a < 3; ++a) {
                        c[a] = cc[a] >> shn;
                        p[a] = qv[a];
                    }
                    L = Ln;
                }
                double vv[3] = {X[0] - o[0], X[1] - o[1], X[2] - o[2]};
                double cx = vv[1] * d64[2] - vv[2] * d64[1], cy = vv[2] * d64[0] - vv[0] * d64[2],
                       cz = vv[0] * d64[1] - vv[1] * d64[0];
                double dt = vv[0] * d64[0] + vv[1] * d64[1] + vv[2] * d64[2];
                angle = atan2(sqrt(cx * cx + cy * cy + cz * cz), dt) * 57.29577951308232;
            }
            steps_out[cm->out_offset_px + local] = steps;
            angle_out[cm->out_offset_px + local] = angle;
        }
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
