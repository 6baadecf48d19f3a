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
#include <numeric>

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

struct Prim {
    Box box;
    float c[3];
};

// Binary node of the first pass: both children's (widened) boxes and refs.
struct BinNode {
    Box box[2];
    int ref[2];
};

struct Builder {
    const float* verts;
    const uint32_t* tris;
    const uint32_t* tri_mat;
    std::vector<Prim> prims;
    std::vector<uint32_t> idx;
    HostBvh* out;
    std::vector<BinNode> bin;
    int max_depth_seen = 0;

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
        for (uint32_t i = b; i < e; ++i) r.grow(prims[idx[i]].box);
        return r;
    }

    int make_leaf(uint32_t b, uint32_t e) {
        uint32_t first = (uint32_t)out->tris.size();
        for (uint32_t i = b; i < e; ++i) {
            uint32_t t = idx[i];
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
            out->tris.push_back(r);
        }
        return ~(int)((first << 3) | (e - b - 1));
    }

    // Returns the child ref of range [b, e).
    int build(uint32_t b, uint32_t e, int depth) {
        uint32_t n = e - b;
        max_depth_seen = std::max(max_depth_seen, depth);
        Box bounds = range_box(b, e);
        Box cb;
        for (uint32_t i = b; i < e; ++i) cb.grow(prims[idx[i]].c);
        double leaf_cost = (double)n;
        int best_axis = -1, best_bin = -1;
        double best_cost = INFINITY;
        constexpr int kBins = 16;
        if (n > 1) {
            for (int ax = 0; ax < 3; ++ax) {
                float ext = cb.hi[ax] - cb.lo[ax];
                if (!(ext > 0.0f)) continue;
                Box bb[kBins];
                uint32_t cnt[kBins] = {};
                float scale = kBins / ext;
                for (uint32_t i = b; i < e; ++i) {
                    const Prim& p = prims[idx[i]];
                    int k = std::min(kBins - 1, (int)((p.c[ax] - cb.lo[ax]) * scale));
                    bb[k].grow(p.box);
                    cnt[k]++;
                }
                double ra[kBins];
                uint32_t rc[kBins];
                Box acc;
                uint32_t c = 0;
                for (int k = kBins - 1; k > 0; --k) {
                    acc.grow(bb[k]);
                    c += cnt[k];
                    ra[k] = acc.area();
                    rc[k] = c;
                }
                Box la;
                uint32_t lc = 0;
                for (int k = 0; k < kBins - 1; ++k) {
                    la.grow(bb[k]);
                    lc += cnt[k];
                    if (lc == 0 || rc[k + 1] == 0) continue;
                    double cost = 1.0 + (la.area() * lc + ra[k + 1] * rc[k + 1]) / std::max(bounds.area(), 1e-30);
                    if (cost < best_cost) {
                        best_cost = cost;
                        best_axis = ax;
                        best_bin = k;
                    }
                }
            }
        }
        bool must_split = n > (uint32_t)kLeafMax;
        if (!must_split && (best_axis < 0 || best_cost >= leaf_cost)) return make_leaf(b, e);
        if (depth >= kMaxBvhDepth - 1) {
            if (!must_split) return make_leaf(b, e);
        }
        uint32_t mid;
        if (best_axis >= 0) {
            float scale = kBins / (cb.hi[best_axis] - cb.lo[best_axis]);
            float lo = cb.lo[best_axis];
            int ax = best_axis, bin = best_bin;
            auto it = std::partition(idx.begin() + b, idx.begin() + e, [&](uint32_t t) {
                int k = std::min(kBins - 1, (int)((prims[t].c[ax] - lo) * scale));
                return k <= bin;
            });
            mid = (uint32_t)(it - idx.begin());
            if (mid == b || mid == e) mid = b + n / 2;
        } else {
            mid = b + n / 2;  // all centroids coincide
        }
        int me = (int)bin.size();
        bin.push_back(BinNode{});
        int l = build(b, mid, depth + 1);
        int r = build(mid, e, depth + 1);
        Box lb = range_box(b, mid), rb = range_box(mid, e);
        widen(lb);
        widen(rb);
        bin[me].box[0] = lb;
        bin[me].box[1] = rb;
        bin[me].ref[0] = l;
        bin[me].ref[1] = r;
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
    }
    B.idx.resize(n_tris);
    std::iota(B.idx.begin(), B.idx.end(), 0u);
    B.bin.reserve(n_tris);
    out->tris.reserve(n_tris);
    const int root2 = B.build(0, n_tris, 0);
    if (B.max_depth_seen >= kMaxBvhDepth) {
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
