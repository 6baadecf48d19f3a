// Host BVH builder: a binary tree by the binned surface-area heuristic (Wald,
// "On fast construction of SAH-based bounding volume hierarchies", RT'07), 16
// bins per axis, leaves of at most kLeafMax triangles; then collapsed into a
// 4-wide tree: a node takes the two children of a binary node and keeps
// opening its largest-area inner child until it holds 4 children or only
// leaves.  Nodes are emitted depth first.  The paper renders with pbrt/lmc;
// the acceleration structure is this library's own.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <future>
#include <system_error>
#include <thread>

#include "jr_internal.h"

namespace jr {
namespace {

struct Box {
    float lo[3] = {INFINITY, INFINITY, INFINITY};
    float hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    void grow(const Box& b) {
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], b.lo[k]);
            hi[k] = std::max(hi[k], b.hi[k]);
        }
    }
    void grow(const float* p) {
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], p[k]);
            hi[k] = std::max(hi[k], p[k]);
        }
    }
    bool empty() const { return lo[0] > hi[0]; }
    double area() const {
        if (empty()) return 0.0;
        double dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
        return 2.0 * (dx * dy + dy * dz + dz * dx);
    }
};

// A triangle's box and centroid, and its index; the build partitions these
// records in place, so every pass reads them in order.
struct Prim {
    Box box;
    float c[3];
    uint32_t id;
};

// Binary node of the first pass: both children's (widened) boxes and refs.
struct BinNode {
    Box box[2];
    int ref[2];
};

// Subtrees of at least this many triangles, this close to the root, are
// built on their own thread (the left one; the right one on the caller's).
constexpr uint32_t kParallelMin = 1024;
constexpr int kParallelDepth = 8;

// A range of at least two chunks of this many prims is binned, and the prims
// of the whole scene set up, by several threads, one chunk range each; the
// chunks' results are merged in order.  Bins and boxes are minima, maxima and
// counts, which do not depend on the order, so the tree is the same.
constexpr uint32_t kChunk = 8192;

constexpr int kBins = 16;

// The bins of a range on the three axes: boxes, counts, and a mask per axis of
// the bins that hold prims.
struct Bins {
    Box bb[3][kBins];
    uint32_t cnt[3][kBins] = {};
    uint32_t used[3] = {0u, 0u, 0u};
    void merge(const Bins& o) {
        for (int ax = 0; ax < 3; ++ax) {
            for (int k = 0; k < kBins; ++k) {
                bb[ax][k].grow(o.bb[ax][k]);
                cnt[ax][k] += o.cnt[ax][k];
            }
            used[ax] |= o.used[ax];
        }
    }
};

uint32_t worker_count(uint32_t n) {
    if (n < 2 * kChunk) return 1u;  // before the query, which may read a file
    return std::min(std::max(1u, std::thread::hardware_concurrency()), n / kChunk);
}

// Runs body(0, chunks) .. body(chunks - 1, chunks): all but the first on
// threads of their own where one can be had, the rest on the caller's.
template <class F>
void run_chunks(uint32_t chunks, F&& body) {
    std::vector<std::future<void>> fut;
    fut.reserve(chunks);
    for (uint32_t c = 1; c < chunks; ++c) {
        try {
            fut.push_back(std::async(std::launch::async, [&body, c, chunks] { body(c, chunks); }));
        } catch (const std::system_error&) {  // no thread to be had: run it here
            body(c, chunks);
        }
    }
    body(0, chunks);
    for (auto& f : fut) f.get();
}

struct Builder {
    const float* verts;
    const uint32_t* tris;
    const uint32_t* tri_mat;
    std::vector<Prim> prims;
    // The binary tree.  The inner node that splits [b, e) at mid is bin[mid - 1]:
    // a split position separates two neighbouring prims for good, so no two
    // nodes share one, and threads building disjoint ranges write disjoint
    // slots.  Positions inside leaves stay unused; collapse() follows refs.
    std::vector<BinNode> bin;
    // Leaf records.  A depth-first build emits the leaves of [b, e) after
    // those of every range left of b, which hold exactly b prims, so the leaf
    // of [b, e) owns records [b, e): the order a single thread would give.
    std::vector<TriRecord> recs;
    HostBvh* out;  // collapse() writes the 4-wide nodes here

    // Widen a box so that a FP32 slab test never rejects a box whose triangle
    // the ray/triangle test accepts (coordinates are rounded outward by a
    // relative 2^-20 plus an absolute 2^-30).
    static void widen(Box& b) {
        for (int k = 0; k < 3; ++k) {
            b.lo[k] = b.lo[k] - (std::fabs(b.lo[k]) * 9.5367431640625e-7f + 9.313225746154785e-10f);
            b.hi[k] = b.hi[k] + (std::fabs(b.hi[k]) * 9.5367431640625e-7f + 9.313225746154785e-10f);
        }
    }

    Box range_box(uint32_t b, uint32_t e) const {
        Box r;
        for (uint32_t i = b; i < e; ++i) r.grow(prims[i].box);
        return r;
    }

    int make_leaf(uint32_t b, uint32_t e) {
        for (uint32_t i = b; i < e; ++i) {
            uint32_t t = prims[i].id;
            const float* v0 = verts + 3 * tris[3 * t];
            const float* v1 = verts + 3 * tris[3 * t + 1];
            const float* v2 = verts + 3 * tris[3 * t + 2];
            TriRecord r;
            int id = (int)t, mat = (int)tri_mat[t];
            float fid, fmat;
            std::memcpy(&fid, &id, 4);
            std::memcpy(&fmat, &mat, 4);
            r.v0_id = make_float4(v0[0], v0[1], v0[2], fid);
            r.e1_mat = make_float4(v1[0] - v0[0], v1[1] - v0[1], v1[2] - v0[2], fmat);
            r.e2 = make_float4(v2[0] - v0[0], v2[1] - v0[1], v2[2] - v0[2], 0.0f);
            recs[i] = r;
        }
        return ~(int)((b << 3) | (e - b - 1));
    }

    // Adds prims [b, e) to the bins of every live axis (centroid box lower
    // corner lo, bins per unit length scale).
    void bin_range(uint32_t b, uint32_t e, const float* lo, const float* scale, const bool* live, Bins& out) const {
        for (uint32_t i = b; i < e; ++i) {
            const Prim& p = prims[i];
            for (int ax = 0; ax < 3; ++ax) {
                if (!live[ax]) continue;
                const int k = std::min(kBins - 1, (int)((p.c[ax] - lo[ax]) * scale[ax]));
                out.bb[ax][k].grow(p.box);
                out.cnt[ax][k]++;
                out.used[ax] |= 1u << k;
            }
        }
    }

    // Returns the child ref of range [b, e); bounds is the range's box, cb the
    // box of its centroids, and max_depth gets the deepest level reached.  One
    // pass bins all three axes; the partition pass also gathers the two sides'
    // centroid boxes, and the sides' boxes come from the chosen split's bins
    // (min and max are exact, so these are the boxes a pass over each side
    // would give).
    int build(uint32_t b, uint32_t e, int depth, const Box& bounds, const Box& cb, int& max_depth) {
        const uint32_t n = e - b;
        max_depth = std::max(max_depth, depth);
        const double leaf_cost = (double)n;
        int best_axis = -1, best_bin = -1;
        double best_cost = INFINITY;
        Bins bins;
        Box (&bb)[3][kBins] = bins.bb;
        uint32_t (&cnt)[3][kBins] = bins.cnt;
        float scale[3] = {0.f, 0.f, 0.f};
        bool live[3] = {false, false, false};
        if (n > 1) {
            for (int ax = 0; ax < 3; ++ax) {
                const float ext = cb.hi[ax] - cb.lo[ax];
                live[ax] = ext > 0.0f;
                if (live[ax]) scale[ax] = kBins / ext;
            }
            const uint32_t chunks = worker_count(n);
            if (chunks == 1) {
                bin_range(b, e, cb.lo, scale, live, bins);
            } else {
                std::vector<Bins> part(chunks);
                run_chunks(chunks, [&](uint32_t c, uint32_t m) {
                    Bins local;  // the chunks' bins in one array would share cache lines at their edges
                    bin_range(b + (uint32_t)((uint64_t)n * c / m), b + (uint32_t)((uint64_t)n * (c + 1) / m), cb.lo,
                              scale, live, local);
                    part[c] = local;
                });
                for (const Bins& q : part) bins.merge(q);
            }
            const double inv_area = 1.0 / std::max(bounds.area(), 1e-30);
            for (int ax = 0; ax < 3; ++ax) {
                if (!live[ax]) continue;
                // Only the bins that hold prims are visited: an empty bin
                // changes neither side's box nor its count, so the candidate
                // after it equals the one before (costs are compared
                // strictly, so the choice is unchanged).  ra[j], rc[j]: area
                // and count of the bins from kept[j] up.
                int kept[kBins], m = 0;
                for (uint32_t u = bins.used[ax]; u; u &= u - 1) kept[m++] = __builtin_ctz(u);
                double ra[kBins];
                uint32_t rc[kBins];
                Box acc;
                uint32_t c = 0;
                for (int j = m - 1; j > 0; --j) {
                    acc.grow(bb[ax][kept[j]]);
                    c += cnt[ax][kept[j]];
                    ra[j] = acc.area();
                    rc[j] = c;
                }
                Box la;
                uint32_t lc = 0;
                for (int j = 0; j + 1 < m; ++j) {
                    la.grow(bb[ax][kept[j]]);
                    lc += cnt[ax][kept[j]];
                    const double cost = 1.0 + (la.area() * lc + ra[j + 1] * rc[j + 1]) * inv_area;
                    if (cost < best_cost) {
                        best_cost = cost;
                        best_axis = ax;
                        best_bin = kept[j];
                    }
                }
            }
        }
        const bool must_split = n > (uint32_t)kLeafMax;
        if (!must_split && (best_axis < 0 || best_cost >= leaf_cost)) return make_leaf(b, e);
        if (depth >= kMaxBvhDepth - 1) {
            if (!must_split) return make_leaf(b, e);
        }
        uint32_t mid = b;
        Box lb, rb, lcb, rcb;
        if (best_axis >= 0) {
            const int ax = best_axis, bin = best_bin;
            const float lo = cb.lo[ax], sc = scale[ax];
            uint32_t i = b, j = e;  // [b, i) left, [j, e) right
            while (i < j) {
                const Prim& p = prims[i];
                if (std::min(kBins - 1, (int)((p.c[ax] - lo) * sc)) <= bin) {
                    lcb.grow(p.c);
                    ++i;
                } else {
                    rcb.grow(p.c);
                    std::swap(prims[i], prims[--j]);
                }
            }
            mid = i;
            for (int k = 0; k <= bin; ++k) lb.grow(bb[ax][k]);
            for (int k = bin + 1; k < kBins; ++k) rb.grow(bb[ax][k]);
        }
        if (best_axis < 0 || mid == b || mid == e) {  // all centroids coincide: split by position
            mid = b + n / 2;
            lb = range_box(b, mid);
            rb = range_box(mid, e);
            lcb = Box();
            rcb = Box();
            for (uint32_t i = b; i < mid; ++i) lcb.grow(prims[i].c);
            for (uint32_t i = mid; i < e; ++i) rcb.grow(prims[i].c);
        }
        int l, r;
        std::future<int> left;
        int left_depth = 0;
        if (n >= kParallelMin && depth < kParallelDepth) {  // the two sides touch disjoint prims and slots
            try {
                left = std::async(std::launch::async,
                                  [&] { return build(b, mid, depth + 1, lb, lcb, left_depth); });
            } catch (const std::system_error&) {  // no thread to be had: both sides here
            }
        }
        if (left.valid()) {
            r = build(mid, e, depth + 1, rb, rcb, max_depth);
            l = left.get();
            max_depth = std::max(max_depth, left_depth);
        } else {
            l = build(b, mid, depth + 1, lb, lcb, max_depth);
            r = build(mid, e, depth + 1, rb, rcb, max_depth);
        }
        widen(lb);
        widen(rb);
        const int me = (int)mid - 1;
        BinNode& nd = bin[me];
        nd.box[0] = lb;
        nd.box[1] = rb;
        nd.ref[0] = l;
        nd.ref[1] = r;
        return me;
    }

    // 4-wide node for binary inner node `b`; returns its index.  `need` gets
    // the most stack entries a traversal below it can hold (a visit pushes at
    // most children - 1 refs), `depth4` the height of its subtree.
    int collapse(int b, int& need, int& depth4) {
        struct Kid {
            int ref;
            Box box;
        };
        Kid kids[4] = {{bin[b].ref[0], bin[b].box[0]}, {bin[b].ref[1], bin[b].box[1]}};
        int n = 2;
        while (n < 4) {
            int pick = -1;
            double best = -1.0;
            for (int j = 0; j < n; ++j)
                if (kids[j].ref >= 0 && kids[j].box.area() > best) {
                    best = kids[j].box.area();
                    pick = j;
                }
            if (pick < 0) break;
            const BinNode& o = bin[kids[pick].ref];
            kids[pick] = {o.ref[0], o.box[0]};
            kids[n++] = {o.ref[1], o.box[1]};
        }
        const int me = (int)out->nodes.size();
        out->nodes.push_back(Bvh4Node{});
        int refs[4] = {kNoChild, kNoChild, kNoChild, kNoChild};
        int sub_need = 0, sub_depth = 0;
        for (int j = 0; j < n; ++j) {
            if (kids[j].ref >= 0) {
                int nd = 0, dp = 0;
                refs[j] = collapse(kids[j].ref, nd, dp);
                sub_need = std::max(sub_need, nd);
                sub_depth = std::max(sub_depth, dp);
            } else {
                refs[j] = kids[j].ref;
            }
        }
        need = (n - 1) + sub_need;
        depth4 = 1 + sub_depth;
        Bvh4Node& q = out->nodes[me];
        float lo[3][4], hi[3][4];
        // an empty slot gets the empty box (lo = +inf, hi = -inf): its entry
        // distance is +inf and its exit distance -inf whatever the ray, so the
        // slab test misses it without looking at the ref
        for (int j = 0; j < 4; ++j)
            for (int k = 0; k < 3; ++k) {
                lo[k][j] = j < n ? kids[j].box.lo[k] : INFINITY;
                hi[k][j] = j < n ? kids[j].box.hi[k] : -INFINITY;
            }
        q.lox = make_float4(lo[0][0], lo[0][1], lo[0][2], lo[0][3]);
        q.hix = make_float4(hi[0][0], hi[0][1], hi[0][2], hi[0][3]);
        q.loy = make_float4(lo[1][0], lo[1][1], lo[1][2], lo[1][3]);
        q.hiy = make_float4(hi[1][0], hi[1][1], hi[1][2], hi[1][3]);
        q.loz = make_float4(lo[2][0], lo[2][1], lo[2][2], lo[2][3]);
        q.hiz = make_float4(hi[2][0], hi[2][1], hi[2][2], hi[2][3]);
        q.refs = make_int4(refs[0], refs[1], refs[2], refs[3]);
        q.pad = make_int4(n, 0, 0, 0);
        return me;
    }
};

}  // namespace

bool build_bvh(const float* verts, uint32_t n_verts, const uint32_t* tris, uint32_t n_tris, const uint32_t* tri_mat,
               HostBvh* out, std::string* err) {
    out->nodes.clear();
    out->tris.clear();
    out->depth = 0;
    if (n_tris == 0) {
        out->root = INT32_MIN;
        return true;
    }
    if (n_tris >= (1u << 27)) {
        *err = "too many triangles (limit 2^27)";
        return false;
    }
    Builder B;
    B.verts = verts;
    B.tris = tris;
    B.tri_mat = tri_mat;
    B.out = out;
    B.prims.resize(n_tris);
    B.bin.resize(n_tris - 1);
    B.recs.resize(n_tris);
    // Each chunk of triangles gets its prims, the box of their boxes and of
    // their centroids, and its first error (1: vertex index out of range, 2:
    // a coordinate not finite); the first chunk with an error names it.
    struct Setup {
        Box box, c;
        int error = 0;
    };
    const uint32_t chunks = worker_count(n_tris);
    std::vector<Setup> part(chunks);
    run_chunks(chunks, [&](uint32_t c, uint32_t m) {
        Setup r;  // local: the chunks' results share cache lines
        const uint32_t t0 = (uint32_t)((uint64_t)n_tris * c / m), t1 = (uint32_t)((uint64_t)n_tris * (c + 1) / m);
        for (uint32_t t = t0; t < t1 && !r.error; ++t) {
            Prim& p = B.prims[t];
            for (int j = 0; j < 3; ++j) {
                const uint32_t vi = tris[3 * t + j];
                if (vi >= n_verts) {
                    r.error = 1;
                    break;
                }
                const float* q = verts + 3 * (size_t)vi;
                if (!std::isfinite(q[0]) || !std::isfinite(q[1]) || !std::isfinite(q[2])) {
                    r.error = 2;
                    break;
                }
                p.box.grow(q);
            }
            for (int k = 0; k < 3; ++k) p.c[k] = 0.5f * (p.box.lo[k] + p.box.hi[k]);
            p.id = t;
            r.box.grow(p.box);
            r.c.grow(p.c);
        }
        part[c] = r;
    });
    Box all_box, all_c;
    for (const Setup& r : part) {
        if (r.error) {
            *err = r.error == 1 ? "triangle vertex index out of range" : "triangle vertex coordinate not finite";
            return false;
        }
        all_box.grow(r.box);
        all_c.grow(r.c);
    }
    int max_depth = 0;
    const int root2 = B.build(0, n_tris, 0, all_box, all_c, max_depth);
    out->tris = std::move(B.recs);
    if (max_depth >= kMaxBvhDepth) {
        *err = "BVH too deep for the traversal stack";
        return false;
    }
    if (root2 < 0) {  // the whole scene is one leaf
        out->root = root2;
        out->depth = 0;
        return true;
    }
    out->nodes.reserve(B.bin.size() / 2 + 1);
    int need = 0, depth4 = 0;
    out->root = B.collapse(root2, need, depth4);
    out->depth = depth4;
    if (need + 1 > kStackSize) {
        *err = "BVH needs more traversal stack than the kernels hold";
        return false;
    }
    return true;
}

}  // namespace jr
