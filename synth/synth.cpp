// Seeded synthetic canvases: stroke-built deep octrees (input generator).
//
// This file builds the inputs that both the CUDA renderer and the FP64 oracle
// consume. It holds none of the ray-casting arithmetic. It implements:
//   * SplitMix64 (Steele, Lea, Flood 2014) uniform doubles from the top 53 bits;
//   * log-uniform draws exp(ln a + u (ln b - ln a)) with the host libm;
//   * spherical brush stamps applied to an adaptive octree: refine down to the
//     cell size that gives about ten cells per brush radius (Sec. 5.2), paint
//     whole cells that lie inside the sphere, paint finest partially covered
//     cells by their centre;
//   * the additive blend of Sec. 5.1: rgb' = B m + (1-m) C, m = B_a/(B_a+C_a),
//     a' = B_a + C_a, evaluated in FP32 with no contraction;
//   * FP16 quantisation (round to nearest even), merge of eight bit-identical
//     sibling leaves (conservative coarsening, Sec. 5.2), and breadth-first
//     canonical record order.
//
// Canonical pool layout (Sec. 4.1.1: index-based pools, eight children per
// allocation unit). Record r has eight int32 slots, child k = x + 2y + 4z
// (Sec. 4.1.1: in its quadtree example the cell above the first child is at offset 2, so +2 is y):
//   slot > 0  : index of the child's record (always > r, breadth-first order)
//   slot == 0 : empty leaf (extinction 0)
//   slot < 0  : a stored leaf of the leaf pool of 4 x FP16 (R,G,B,sigma). Leaves are numbered
//               0, 1, ... in breadth-first slot order, and the slot holds -(number mod 2^31) - 1,
//               so pools can pass 2^31 leaves with 32-bit slots (below 2^31, -slot-1 is the number).
// Record 0 is the root cell [-E/2, E/2]^3.
#include <cstdint>
#include <cstring>
#include <cmath>
#include <vector>
#include <array>
#include <deque>
#include <algorithm>
#include <atomic>
#include <thread>

namespace {

struct Tree {
    int32_t D = 0;
    double E = 0.0;
    std::vector<std::array<int32_t, 8>> rec;   // building records
    std::vector<std::array<float, 4>> val;     // FP32 leaf accumulators (r,g,b,sigma)
    // finalize outputs
    std::vector<int32_t> out_nodes;
    std::vector<uint16_t> out_leaves;
    int32_t max_level = 0;
};

struct Stamp {
    double c[3];
    double r, r2;
    float rgba[4];
    int32_t kt;  // target depth
};

// FP32 additive blend of the brush B into the canvas value C (Sec. 5.1).
inline void blend(std::array<float, 4>& C, const float B[4]) {
    const float s = B[3] + C[3];
    if (s == 0.0f) return;
    float m = B[3] / s;
    float om = 1.0f - m;
    for (int i = 0; i < 3; ++i) {
        float a = B[i] * m;
        float b = om * C[i];
        C[i] = a + b;
    }
    C[3] = s;
}

int32_t new_leaf(Tree& T, const std::array<float, 4>& v) {
    T.val.push_back(v);
    return -(int32_t)T.val.size();   // leaf index = size-1 -> slot = -(idx+1)
}

void paint_all_slot(Tree& T, int32_t rec, int k, const Stamp& s) {
    int32_t v = T.rec[rec][k];
    if (v > 0) {
        for (int j = 0; j < 8; ++j) paint_all_slot(T, v, j, s);
    } else if (v == 0) {
        std::array<float, 4> z = {0.f, 0.f, 0.f, 0.f};
        blend(z, s.rgba);
        int32_t nv = new_leaf(T, z);
        T.rec[rec][k] = nv;
    } else {
        blend(T.val[-v - 1], s.rgba);
    }
}

inline double sq(double x) { return x * x; }

void paint_rec(Tree& T, int32_t rec, int32_t level, double lx, double ly, double lz, double size, const Stamp& s);

// Squared distances from the sphere centre to the box [b, b+h]^3 and to its farthest corner.
inline void box_dist2(const Stamp& s, double bx, double by, double bz, double h, double& dmin2, double& dmax2) {
    dmin2 = 0.0;
    dmax2 = 0.0;
    const double lo[3] = {bx, by, bz};
    for (int a = 0; a < 3; ++a) {
        const double c = s.c[a];
        const double l = lo[a], u = lo[a] + h;
        if (c < l) dmin2 += sq(l - c);
        else if (c > u) dmin2 += sq(c - u);
        dmax2 += std::fmax(sq(c - l), sq(u - c));
    }
}

// Apply stamp s to slot k of record rec; the slot is a cell at level cl with box [b, b+h]^3.
void paint_child(Tree& T, int32_t rec, int k, int32_t cl, double bx, double by, double bz, double h, const Stamp& s) {
    double dmin2, dmax2;
    box_dist2(s, bx, by, bz, h, dmin2, dmax2);
    if (dmin2 >= s.r2) return;                                  // outside
    if (dmax2 <= s.r2) { paint_all_slot(T, rec, k, s); return; }  // inside: painted whole
    int32_t v = T.rec[rec][k];
    if (v > 0) { paint_rec(T, v, cl, bx, by, bz, h, s); return; }
    if (cl < s.kt && cl < T.D) {
        // refine the leaf: eight children copy its value (Sec. 4.1.1: always eight)
        std::array<int32_t, 8> kids;
        if (v == 0) {
            kids.fill(0);
        } else {
            std::array<float, 4> pv = T.val[-v - 1];
            for (int j = 0; j < 8; ++j) kids[j] = new_leaf(T, pv);
        }
        T.rec.push_back(kids);
        int32_t nr = (int32_t)T.rec.size() - 1;
        T.rec[rec][k] = nr;
        paint_rec(T, nr, cl, bx, by, bz, h, s);
        return;
    }
    // finest partially covered cell: painted iff its centre is inside
    const double d2 = sq(bx + 0.5 * h - s.c[0]) + sq(by + 0.5 * h - s.c[1]) + sq(bz + 0.5 * h - s.c[2]);
    if (d2 < s.r2) paint_all_slot(T, rec, k, s);
}

void paint_rec(Tree& T, int32_t rec, int32_t level, double lx, double ly, double lz, double size, const Stamp& s) {
    const double h = size * 0.5;
    for (int k = 0; k < 8; ++k)
        paint_child(T, rec, k, level + 1, lx + ((k & 1) ? h : 0.0), ly + ((k & 2) ? h : 0.0), lz + ((k & 4) ? h : 0.0), h, s);
}

// IEEE binary16 bits of x, round to nearest even (through the compiler's _Float16).
inline uint16_t to_half_bits(float x) {
    _Float16 h = (_Float16)x;
    uint16_t b;
    std::memcpy(&b, &h, 2);
    return b;
}

}  // namespace

extern "C" {

// SplitMix64: state advances by the golden gamma; output mixed by two multiply-xorshift rounds.
void synth_splitmix_uniform(uint64_t* state, int64_t n, double* out) {
    uint64_t s = *state;
    for (int64_t i = 0; i < n; ++i) {
        s += 0x9E3779B97F4A7C15ull;
        uint64_t z = s;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z = z ^ (z >> 31);
        out[i] = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    }
    *state = s;
}

void synth_log_uniform(double a, double b, const double* u, int64_t n, double* out) {
    const double la = std::log(a), lb = std::log(b);
    for (int64_t i = 0; i < n; ++i) out[i] = std::exp(la + u[i] * (lb - la));
}

}  // extern "C"

namespace {

// ---------------------------------------------------------------------------
// Builder: stamps are collected, then painted in parallel over a spatial
// partition. A partition cell is pre-refined only when every stamp that
// partially covers it would refine it anyway (its target depth is deeper than
// the cell), so each partition leaf evolves exactly as in one sequential pass
// over the ordered stamps, and the canonical merged tree is the same.
// ---------------------------------------------------------------------------
struct PNode {
    int32_t level = 0;
    double lo[3] = {0, 0, 0};
    double size = 0;
    std::vector<int32_t> st;
    int32_t kid[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
    bool leaf = true;
    int64_t ckey = -1;
    Tree local;
    std::vector<uint64_t> key;
    std::vector<int64_t> coll;
};

struct Builder {
    int32_t D;
    double E;
    std::vector<Stamp> stamps;
    std::vector<PNode> P;
    int64_t n_rec = 0, n_leaf = 0;
    int32_t levels = 0;
    int32_t root_levels = 1;  // levels kept refined everywhere (2: the 4^3 array of roots of Sec. 4)
    bool finalized = false;
};

int g_threads = 0;
int32_t g_split = 512;

void build_partition(Builder& B, int32_t p) {
    B.P[p].leaf = false;
    const double h = B.P[p].size * 0.5;
    for (int k = 0; k < 8; ++k) {
        PNode c;
        c.level = B.P[p].level + 1;
        c.size = h;
        c.lo[0] = B.P[p].lo[0] + ((k & 1) ? h : 0.0);
        c.lo[1] = B.P[p].lo[1] + ((k & 2) ? h : 0.0);
        c.lo[2] = B.P[p].lo[2] + ((k & 4) ? h : 0.0);
        bool can_split = c.level < B.D;
        for (int32_t si : B.P[p].st) {
            const Stamp& s = B.stamps[si];
            double dmin2, dmax2;
            box_dist2(s, c.lo[0], c.lo[1], c.lo[2], h, dmin2, dmax2);
            if (dmin2 >= s.r2) continue;
            c.st.push_back(si);
            if (dmax2 > s.r2 && !(s.kt > c.level)) can_split = false;
        }
        const bool split = can_split && (int32_t)c.st.size() > g_split;
        int32_t ci = (int32_t)B.P.size();
        B.P.push_back(std::move(c));
        B.P[p].kid[k] = ci;
        if (split) build_partition(B, ci);
    }
    std::vector<int32_t>().swap(B.P[p].st);
}

void paint_partition_leaf(Builder& B, PNode& N) {
    N.local.D = B.D;
    N.local.E = B.E;
    std::array<int32_t, 8> pseudo;
    pseudo.fill(0);
    N.local.rec.push_back(pseudo);  // record 0 holds this cell in slot 0
    for (int32_t si : N.st) paint_child(N.local, 0, 0, N.level, N.lo[0], N.lo[1], N.lo[2], N.size, B.stamps[si]);
    std::vector<int32_t>().swap(N.st);
    // quantise to FP16 keys (0 = empty) and collapse uniform subtrees (reverse index order is post-order)
    N.key.resize(N.local.val.size());
    for (size_t i = 0; i < N.local.val.size(); ++i) {
        const auto& v = N.local.val[i];
        float r = std::fmin(std::fmax(v[0], 0.0f), 1.0f);
        float g = std::fmin(std::fmax(v[1], 0.0f), 1.0f);
        float b = std::fmin(std::fmax(v[2], 0.0f), 1.0f);
        float a = std::fmin(std::fmax(v[3], 0.0f), 60000.0f);
        uint16_t ha = to_half_bits(a);
        N.key[i] = ha == 0 ? 0 : ((uint64_t)to_half_bits(r) | ((uint64_t)to_half_bits(g) << 16) |
                                  ((uint64_t)to_half_bits(b) << 32) | ((uint64_t)ha << 48));
    }
    std::vector<std::array<float, 4>>().swap(N.local.val);
    const size_t nr = N.local.rec.size();
    N.coll.assign(nr, -1);
    for (size_t ri = nr; ri-- > 1;) {
        auto sk = [&](int32_t v) -> int64_t { return v == 0 ? 0 : (v < 0 ? (int64_t)N.key[-v - 1] : N.coll[v]); };
        int64_t k0 = sk(N.local.rec[ri][0]);
        if (k0 < 0) continue;
        bool same = true;
        for (int k = 1; k < 8 && same; ++k) same = (sk(N.local.rec[ri][k]) == k0);
        if (same) N.coll[ri] = k0;
    }
}

// A resolved slot: internal node handle (tree, rec) or a leaf key.
struct Slot {
    bool internal;
    int32_t tree;  // -1: partition node, else partition-leaf index owning the local record
    int32_t rec;
    uint64_t key;
};

inline Slot local_slot(const PNode& N, int32_t owner, int32_t v) {
    if (v == 0) return {false, 0, 0, 0};
    if (v < 0) return {false, 0, 0, N.key[-v - 1]};
    if (N.coll[v] >= 0) return {false, 0, 0, (uint64_t)N.coll[v]};
    return {true, owner, v, 0};
}

inline Slot resolve(const Builder& B, int32_t tree, int32_t rec, int k) {
    if (tree < 0) {
        const int32_t c = B.P[rec].kid[k];
        const PNode& C = B.P[c];
        if (C.leaf) return local_slot(C, c, C.local.rec[0][0]);
        if (C.ckey >= 0) return {false, 0, 0, (uint64_t)C.ckey};
        return {true, -1, c, 0};
    }
    const PNode& N = B.P[tree];
    return local_slot(N, tree, N.local.rec[rec][k]);
}

int64_t collapse_partition(Builder& B, int32_t p) {
    int64_t k0 = -2;
    bool same = true;
    for (int k = 0; k < 8; ++k) {
        const int32_t c = B.P[p].kid[k];
        if (!B.P[c].leaf) collapse_partition(B, c);
        Slot s = resolve(B, -1, p, k);
        int64_t kk = s.internal ? -1 : (int64_t)s.key;
        if (k == 0) k0 = kk;
        else if (kk != k0) same = false;
    }
    B.P[p].ckey = (p != 0 && same && k0 >= 0) ? k0 : -1;
    return B.P[p].ckey;
}

// Breadth-first walk; writes records/leaves when the output pointers are given. Cells above
// level root_levels are always records: a uniform one (tree -2) where the cell is a leaf.
int bfs(Builder& B, int32_t* nodes, uint16_t* leaves, int64_t* n_rec, int64_t* n_leaf, int32_t* levels) {
    std::deque<std::pair<std::pair<int32_t, int32_t>, int32_t>> q;
    std::vector<uint64_t> uniform;
    q.push_back({{-1, 0}, 0});
    int64_t next_rec = 1, nl = 0, ri = 0;
    int32_t maxl = 1;
    while (!q.empty()) {
        auto [h, lev] = q.front();
        q.pop_front();
        if (lev + 1 > maxl) maxl = lev + 1;
        for (int k = 0; k < 8; ++k) {
            Slot s = h.first == -2 ? Slot{false, 0, 0, uniform[(size_t)h.second]} : resolve(B, h.first, h.second, k);
            int32_t out;
            if (!s.internal && lev + 1 < B.root_levels) {
                out = (int32_t)next_rec++;
                q.push_back({{-2, (int32_t)uniform.size()}, lev + 1});
                uniform.push_back(s.key);
            } else if (s.internal) {
                if (next_rec >= 0x7FFFFFFF) return -1;
                out = (int32_t)next_rec++;
                q.push_back({{s.tree, s.rec}, lev + 1});
            } else if (s.key == 0) {
                out = 0;
            } else {
                if (nl >= ((int64_t)8 << 31)) return -1;  // beyond 2^34 leaves
                out = -(int32_t)(nl & 0x7FFFFFFF) - 1;
                if (leaves)
                    for (int c = 0; c < 4; ++c) leaves[4 * nl + c] = (uint16_t)(s.key >> (16 * c));
                ++nl;
            }
            if (nodes) nodes[8 * ri + k] = out;
        }
        ++ri;
    }
    *n_rec = ri;
    *n_leaf = nl;
    *levels = maxl;
    return 0;
}

}  // namespace

extern "C" {

void synth_set_threads(int32_t n) { g_threads = n; }

// Keep the top n levels refined everywhere (n = 2: a 4^3 array of roots); before finalize.
int synth_tree_set_root_levels(void* h, int32_t n) {
    Builder& B = *static_cast<Builder*>(h);
    if (n < 1 || n >= B.D || B.finalized) return -1;
    B.root_levels = n;
    return 0;
}

// Partition cells holding more than n stamps are split when that is exact (default 512).
void synth_set_split(int32_t n) { g_split = n > 0 ? n : 512; }

void* synth_tree_new(int32_t depth, double extent) {
    if (depth < 1 || depth > 30 || !(extent > 0.0)) return nullptr;
    Builder* B = new Builder();
    B->D = depth;
    B->E = extent;
    return B;
}

void synth_tree_free(void* h) { delete static_cast<Builder*>(h); }

// Queue n spherical stamps (painted in this order at finalize).
// rgba: n x 4 FP32 (R,G,B in [0,1], A = extinction per canvas unit).
int synth_tree_stamp_spheres(void* h, int64_t n, const double* centers, const double* radii, const float* rgba) {
    Builder& B = *static_cast<Builder*>(h);
    if (B.finalized) return -2;
    if ((int64_t)B.stamps.size() + n >= 0x7FFFFFFF) return -1;
    for (int64_t i = 0; i < n; ++i) {
        Stamp s;
        for (int a = 0; a < 3; ++a) s.c[a] = centers[3 * i + a];
        s.r = radii[i];
        s.r2 = s.r * s.r;
        for (int a = 0; a < 4; ++a) s.rgba[a] = rgba[4 * i + a];
        // target depth: smallest k with E 2^-k <= r/10 (integer loop), capped at D
        int32_t k = 0;
        double w = B.E;
        const double tgt = s.r / 10.0;
        while (k < B.D && w > tgt) { w *= 0.5; ++k; }
        s.kt = k;
        B.stamps.push_back(s);
    }
    return 0;
}

// Paint all stamps, quantise, merge identical siblings, count the breadth-first pools.
int synth_tree_finalize(void* h, int64_t* n_records, int64_t* n_leaves, int32_t* max_level) {
    Builder& B = *static_cast<Builder*>(h);
    if (!B.finalized) {
        PNode root;
        root.level = 0;
        root.size = B.E;
        root.lo[0] = root.lo[1] = root.lo[2] = -0.5 * B.E;
        for (int32_t i = 0; i < (int32_t)B.stamps.size(); ++i) {
            double dmin2, dmax2;
            box_dist2(B.stamps[i], root.lo[0], root.lo[1], root.lo[2], root.size, dmin2, dmax2);
            if (dmin2 < B.stamps[i].r2) root.st.push_back(i);
        }
        B.P.reserve(1 << 16);
        B.P.push_back(std::move(root));
        build_partition(B, 0);
        std::vector<int32_t> leaves;
        for (int32_t i = 0; i < (int32_t)B.P.size(); ++i)
            if (B.P[i].leaf) leaves.push_back(i);
        // largest lists first
        std::sort(leaves.begin(), leaves.end(), [&](int32_t a, int32_t b) { return B.P[a].st.size() > B.P[b].st.size(); });
        int nt = g_threads > 0 ? g_threads : (int)std::thread::hardware_concurrency();
        if (nt < 1) nt = 1;
        std::atomic<size_t> next{0};
        auto work = [&]() {
            for (;;) {
                size_t i = next.fetch_add(1);
                if (i >= leaves.size()) break;
                paint_partition_leaf(B, B.P[leaves[i]]);
            }
        };
        std::vector<std::thread> th;
        for (int t = 1; t < nt; ++t) th.emplace_back(work);
        work();
        for (auto& t : th) t.join();
        collapse_partition(B, 0);
        if (bfs(B, nullptr, nullptr, &B.n_rec, &B.n_leaf, &B.levels) != 0) return -1;
        B.finalized = true;
    }
    *n_records = B.n_rec;
    *n_leaves = B.n_leaf;
    *max_level = B.levels;
    return 0;
}

int synth_tree_export(void* h, int32_t* nodes, uint16_t* leaves) {
    Builder& B = *static_cast<Builder*>(h);
    if (!B.finalized) return -2;
    int64_t a, b;
    int32_t c;
    return bfs(B, nodes, leaves, &a, &b, &c);
}

// Partition statistics and building-tree sizes (records, leaf accumulators).
void synth_tree_sizes(void* h, int64_t* n_build_records, int64_t* n_build_values) {
    Builder& B = *static_cast<Builder*>(h);
    int64_t r = 0, v = 0;
    for (const auto& p : B.P) {
        r += (int64_t)p.local.rec.size();
        v += (int64_t)p.key.size();
    }
    *n_build_records = r;
    *n_build_values = v;
}

}  // extern "C"
