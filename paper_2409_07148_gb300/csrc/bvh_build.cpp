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

// The output of a (sub)tree build: binary nodes and leaf triangle records in
// depth-first order, refs relative to these arrays.
struct Part {
    std::vector<BinNode> bin;
    std::vector<TriRecord> tris;
    int max_depth = 0;
};

// Append part q after part p, moving q's refs by p's sizes; returns ref moved.
// Appending a node's left and then its right part reproduces the order a
// sequential depth-first build would give.
int append_part(Part& p, Part& q, int ref) {
    const int node_off = (int)p.bin.size(), tri_off = (int)p.tris.size();
    for (BinNode& nd : q.bin)
        for (int j = 0; j < 2; ++j) nd.ref[j] = rebase_ref(nd.ref[j], node_off, tri_off);
    p.bin.insert(p.bin.end(), q.bin.begin(), q.bin.end());
    p.tris.insert(p.tris.end(), q.tris.begin(), q.tris.end());
    p.max_depth = std::max(p.max_depth, q.max_depth);
    return rebase_ref(ref, node_off, tri_off);
}

// Subtrees of at least this many triangles, this close to the root, are
// built on their own thread (the left one; the right one on the caller's).
constexpr uint32_t kParallelMin = 8192;
constexpr int kParallelDepth = 4;

struct Builder {
    const float* verts;
    const uint32_t* tris;
    const uint32_t* tri_mat;
    std::vector<Prim> prims;
    std::vector<BinNode> bin;  // the binary tree, for collapse()
    HostBvh* out;              // collapse() writes the 4-wide nodes here

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

    int make_leaf(uint32_t b, uint32_t e, Part& out) {
        uint32_t first = (uint32_t)out.tris.size();
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
            out.tris.push_back(r);
        }
        return ~(int)((first << 3) | (e - b - 1));
    }

    // Returns the child ref of range [b, e); bounds is the range's box and cb
    // the box of its centroids.  One pass bins all three axes; the partition
    // pass also gathers the two sides' centroid boxes, and the sides' boxes
    // come from the chosen split's bins (min and max are exact, so these are
    // the boxes a pass over each side would give).
    int build(uint32_t b, uint32_t e, int depth, const Box& bounds, const Box& cb, Part& out) {
        const uint32_t n = e - b;
        out.max_depth = std::max(out.max_depth, depth);
        const double leaf_cost = (double)n;
        int best_axis = -1, best_bin = -1;
        double best_cost = INFINITY;
        constexpr int kBins = 16;
        Box bb[3][kBins];
        uint32_t cnt[3][kBins] = {};
        float scale[3] = {0.f, 0.f, 0.f};
        bool live[3] = {false, false, false};
        if (n > 1) {
            for (int ax = 0; ax < 3; ++ax) {
                const float ext = cb.hi[ax] - cb.lo[ax];
                live[ax] = ext > 0.0f;
                if (live[ax]) scale[ax] = kBins / ext;
            }
            for (uint32_t i = b; i < e; ++i) {
                const Prim& p = prims[i];
                for (int ax = 0; ax < 3; ++ax) {
                    if (!live[ax]) continue;
                    const int k = std::min(kBins - 1, (int)((p.c[ax] - cb.lo[ax]) * scale[ax]));
                    bb[ax][k].grow(p.box);
                    cnt[ax][k]++;
                }
            }
            const double inv_area = 1.0 / std::max(bounds.area(), 1e-30);
            for (int ax = 0; ax < 3; ++ax) {
                if (!live[ax]) continue;
                // An empty bin changes neither side's box nor its count: the
                // candidate after it equals the one before, so it is skipped
                // (costs are compared strictly, so the choice is unchanged).
                double ra[kBins];
                uint32_t rc[kBins];
                Box acc;
                uint32_t c = 0;
                double a = 0.0;
                for (int k = kBins - 1; k > 0; --k) {
                    if (cnt[ax][k]) {
                        acc.grow(bb[ax][k]);
                        c += cnt[ax][k];
                        a = acc.area();
                    }
                    ra[k] = a;
                    rc[k] = c;
                }
                Box la;
                uint32_t lc = 0;
                for (int k = 0; k < kBins - 1; ++k) {
                    if (!cnt[ax][k]) continue;
                    la.grow(bb[ax][k]);
                    lc += cnt[ax][k];
                    if (rc[k + 1] == 0) continue;
                    const double cost = 1.0 + (la.area() * lc + ra[k + 1] * rc[k + 1]) * inv_area;
                    if (cost < best_cost) {
                        best_cost = cost;
                        best_axis = ax;
                        best_bin = k;
                    }
                }
            }
        }
        const bool must_split = n > (uint32_t)kLeafMax;
        if (!must_split && (best_axis < 0 || best_cost >= leaf_cost)) return make_leaf(b, e, out);
        if (depth >= kMaxBvhDepth - 1) {
            if (!must_split) return make_leaf(b, e, out);
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
        const int me = (int)out.bin.size();
        out.bin.push_back(BinNode{});
        int l, r;
        Part pl, pr;
        std::future<int> left;
        if (n >= kParallelMin && depth < kParallelDepth) {  // the two sides touch disjoint prims
            try {
                left = std::async(std::launch::async, [&] { return build(b, mid, depth + 1, lb, lcb, pl); });
            } catch (const std::system_error&) {  // no thread to be had: both sides here
            }
        }
        if (left.valid()) {
            const int rr = build(mid, e, depth + 1, rb, rcb, pr);
            const int lr = left.get();
            l = append_part(out, pl, lr);
            r = append_part(out, pr, rr);
        } else {
            l = build(b, mid, depth + 1, lb, lcb, out);
            r = build(mid, e, depth + 1, rb, rcb, out);
        }
        widen(lb);
        widen(rb);
        BinNode& nd = out.bin[me];
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
    for (uint32_t t = 0; t < n_tris; ++t) {
        Prim& p = B.prims[t];
        for (int j = 0; j < 3; ++j) {
            uint32_t vi = tris[3 * t + j];
            if (vi >= n_verts) {
                *err = "triangle vertex index out of range";
                return false;
            }
            p.box.grow(verts + 3 * vi);
        }
        for (int k = 0; k < 3; ++k) p.c[k] = 0.5f * (p.box.lo[k] + p.box.hi[k]);
        p.id = t;
    }
    Part root;
    root.bin.reserve(n_tris);
    root.tris.reserve(n_tris);
    Box all_box, all_c;
    for (uint32_t t = 0; t < n_tris; ++t) {
        all_box.grow(B.prims[t].box);
        all_c.grow(B.prims[t].c);
    }
    const int root2 = B.build(0, n_tris, 0, all_box, all_c, root);
    B.bin = std::move(root.bin);
    out->tris = std::move(root.tris);
    if (root.max_depth >= kMaxBvhDepth) {
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
