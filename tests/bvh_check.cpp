// Host-side check of the BVH builder (bvh_build.cpp), compiled by
// tests/test_bvh_host.py with the host compiler; it runs no GPU code.
//
// Reads a scene (n_verts, n_tris, verts float[3 n_verts], tris u32[3 n_tris],
// materials u32[n_tris]) from argv[1], builds the tree twice and prints one
// line of key=value results.  argv[2] = "shrink" or "drop" first damages the
// tree (the root's first child box loses its x extent; a leaf of two or more
// triangles loses one), so that the test can see the checks fail.
// argv[2] = "merge" with a second scene in argv[3]: both trees are put into one
// pair of arrays as a batch merges its scenes (the second one's nodes and
// records after the first one's, its refs moved by rebase_ref and its
// material indices by the first scene's count), and each scene's part is
// checked from its moved root: merge_a, merge_b = cover, refs, contain and
// records all hold.  "merge_off_by_one" moves the second scene's leaves by one
// record too few, which the check must see.  Results:
//   ok          the builder accepted the scene
//   same        the two builds are byte-identical (the top subtrees are built
//               on separate threads; their merge must not depend on timing)
//   cover       every triangle id appears in exactly one leaf record
//   records     each record holds its triangle's v0, v1 - v0, v2 - v0, material
//   refs        every child ref is an inner node index below the node count, a
//               leaf range inside the records, or the empty-slot marker
//   empty       every empty slot carries the empty box (lo = +inf, hi = -inf)
//   contain     every child box contains every vertex of every triangle below it
//   stack       the deepest stack a traversal can need (child count - 1 summed
//               along a root-to-leaf path) fits the kernels' stack
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "jr_internal.h"

namespace {

struct Scene {
    std::vector<float> v;
    std::vector<uint32_t> t, m;
};

bool read_scene(const char* path, Scene& s) {
    FILE* f = std::fopen(path, "rb");
    if (!f) return false;
    uint32_t nv = 0, nt = 0;
    bool ok = std::fread(&nv, 4, 1, f) == 1 && std::fread(&nt, 4, 1, f) == 1;
    if (ok) {
        s.v.resize(3 * (size_t)nv);
        s.t.resize(3 * (size_t)nt);
        s.m.resize(nt);
        ok = std::fread(s.v.data(), 4, s.v.size(), f) == s.v.size() &&
             std::fread(s.t.data(), 4, s.t.size(), f) == s.t.size() &&
             std::fread(s.m.data(), 4, s.m.size(), f) == s.m.size();
    }
    std::fclose(f);
    return ok;
}

struct Checker {
    const Scene& s;
    const jr::HostBvh& b;
    std::vector<int> seen;
    bool refs = true, empty = true, contain = true;

    // Every vertex of every triangle in the subtree of `ref` lies in the box.
    bool inside(int ref, const float lo[3], const float hi[3]) const {
        if (ref == jr::kNoChild) return true;
        if (ref < 0) {
            const int enc = ~ref, first = enc >> 3, cnt = (enc & 7) + 1;
            for (int k = first; k < first + cnt; ++k) {
                int id;
                const float w = b.tris[k].v0_id.w;
                std::memcpy(&id, &w, 4);
                for (int j = 0; j < 3; ++j) {
                    const float* p = &s.v[3 * (size_t)s.t[3 * (size_t)id + j]];
                    for (int a = 0; a < 3; ++a)
                        if (p[a] < lo[a] || p[a] > hi[a]) return false;
                }
            }
            return true;
        }
        const jr::Bvh4Node& n = b.nodes[ref];
        const int r[4] = {n.refs.x, n.refs.y, n.refs.z, n.refs.w};
        for (int j = 0; j < 4; ++j)
            if (!inside(r[j], lo, hi)) return false;
        return true;
    }

    void leaf(int ref) {
        const int enc = ~ref, first = enc >> 3, cnt = (enc & 7) + 1;
        if (first < 0 || first + cnt > (int)b.tris.size()) {
            refs = false;
            return;
        }
        for (int k = first; k < first + cnt; ++k) {
            int id;
            const float w = b.tris[k].v0_id.w;
            std::memcpy(&id, &w, 4);
            if (id >= 0 && id < (int)seen.size()) seen[id]++;
        }
    }

    // Walks the tree; returns the stack need of the subtree below `ref`.
    int walk(int ref) {
        if (ref == jr::kNoChild) return 0;
        if (ref < 0) {
            leaf(ref);
            return 0;
        }
        if (ref >= (int)b.nodes.size()) {
            refs = false;
            return 0;
        }
        const jr::Bvh4Node& n = b.nodes[ref];
        const float* lo[3] = {&n.lox.x, &n.loy.x, &n.loz.x};
        const float* hi[3] = {&n.hix.x, &n.hiy.x, &n.hiz.x};
        const int r[4] = {n.refs.x, n.refs.y, n.refs.z, n.refs.w};
        int kids = 0, need = 0;
        for (int j = 0; j < 4; ++j) {
            const float l[3] = {lo[0][j], lo[1][j], lo[2][j]}, h[3] = {hi[0][j], hi[1][j], hi[2][j]};
            if (r[j] == jr::kNoChild) {
                for (int a = 0; a < 3; ++a)
                    if (!(l[a] == INFINITY && h[a] == -INFINITY)) empty = false;
                continue;
            }
            ++kids;
            if (!inside(r[j], l, h)) contain = false;
            need = std::max(need, walk(r[j]));
        }
        return kids - 1 + need;
    }
};

}  // namespace

// The checks of one scene's part of a tree whose root is `root`: cover,
// refs, contain, and records (material index moved by mat_off).
bool part_ok(const Scene& s, const jr::HostBvh& t, int root, int mat_off) {
    const uint32_t nt = (uint32_t)s.m.size();
    Checker c{s, t, std::vector<int>(nt, 0)};
    c.walk(root);
    bool ok = c.refs && c.contain && c.empty;
    for (uint32_t k = 0; k < nt && ok; ++k) ok = c.seen[k] == 1;
    // records of this part: the leaves reached from root
    std::vector<int> stack{root};
    while (ok && !stack.empty()) {
        const int ref = stack.back();
        stack.pop_back();
        if (ref == jr::kNoChild) continue;
        if (ref >= 0) {
            const jr::Bvh4Node& n = t.nodes[ref];
            stack.insert(stack.end(), {n.refs.x, n.refs.y, n.refs.z, n.refs.w});
            continue;
        }
        const int enc = ~ref, first = enc >> 3, cnt = (enc & 7) + 1;
        for (int k = first; k < first + cnt && ok; ++k) {
            int id, mat;
            std::memcpy(&id, &t.tris[k].v0_id.w, 4);
            std::memcpy(&mat, &t.tris[k].e1_mat.w, 4);
            const float* p0 = &s.v[3 * (size_t)s.t[3 * (size_t)id]];
            ok = t.tris[k].v0_id.x == p0[0] && t.tris[k].v0_id.y == p0[1] && t.tris[k].v0_id.z == p0[2] &&
                 mat == (int)s.m[id] + mat_off;
        }
    }
    return ok;
}

int merge_main(const Scene& sa, const char* other, bool off_by_one) {
    Scene sb;
    if (!read_scene(other, sb)) {
        std::printf("error=read\n");
        return 2;
    }
    jr::HostBvh a, b;
    std::string err;
    if (!jr::build_bvh(sa.v.data(), (uint32_t)(sa.v.size() / 3), sa.t.data(), (uint32_t)sa.m.size(), sa.m.data(), &a,
                       &err) ||
        !jr::build_bvh(sb.v.data(), (uint32_t)(sb.v.size() / 3), sb.t.data(), (uint32_t)sb.m.size(), sb.m.data(), &b,
                       &err)) {
        std::printf("ok=0 error=%s\n", err.c_str());
        return 0;
    }
    // scene a's materials are numbered 0 .. max + 1 in this check
    int mat_count = 0;
    for (uint32_t m : sa.m) mat_count = std::max(mat_count, (int)m + 1);
    jr::HostBvh m = a;
    const int node_off = (int)a.nodes.size(), tri_off = (int)a.tris.size() - (off_by_one ? 1 : 0);
    for (jr::Bvh4Node n : b.nodes) {
        int* r = &n.refs.x;
        for (int j = 0; j < 4; ++j) r[j] = jr::rebase_ref(r[j], node_off, tri_off);
        m.nodes.push_back(n);
    }
    for (jr::TriRecord r : b.tris) {
        int mat;
        std::memcpy(&mat, &r.e1_mat.w, 4);
        mat += mat_count;
        std::memcpy(&r.e1_mat.w, &mat, 4);
        m.tris.push_back(r);
    }
    const int root_b = jr::rebase_ref(b.root, node_off, tri_off);
    std::printf("ok=1 merge_a=%d merge_b=%d\n", part_ok(sa, m, a.root, 0), part_ok(sb, m, root_b, mat_count));
    return 0;
}

int main(int argc, char** argv) {
    Scene s;
    if (argc < 2 || !read_scene(argv[1], s)) {
        std::printf("error=read\n");
        return 2;
    }
    if (argc > 3 && std::string(argv[2]) == "merge") return merge_main(s, argv[3], false);
    if (argc > 3 && std::string(argv[2]) == "merge_off_by_one") return merge_main(s, argv[3], true);
    const uint32_t nv = (uint32_t)(s.v.size() / 3), nt = (uint32_t)s.m.size();
    jr::HostBvh a, b;
    std::string err;
    const bool ok = jr::build_bvh(s.v.data(), nv, s.t.data(), nt, s.m.data(), &a, &err) &&
                    jr::build_bvh(s.v.data(), nv, s.t.data(), nt, s.m.data(), &b, &err);
    if (!ok) {
        std::printf("ok=0 error=%s\n", err.c_str());
        return 0;
    }
    const bool same = a.root == b.root && a.nodes.size() == b.nodes.size() && a.tris.size() == b.tris.size() &&
                      std::memcmp(a.nodes.data(), b.nodes.data(), sizeof(jr::Bvh4Node) * a.nodes.size()) == 0 &&
                      std::memcmp(a.tris.data(), b.tris.data(), sizeof(jr::TriRecord) * a.tris.size()) == 0;
    bool records = a.tris.size() == nt;
    for (size_t k = 0; k < a.tris.size() && records; ++k) {
        const jr::TriRecord& r = a.tris[k];
        int id, mat;
        std::memcpy(&id, &r.v0_id.w, 4);
        std::memcpy(&mat, &r.e1_mat.w, 4);
        if (id < 0 || id >= (int)nt) {
            records = false;
            break;
        }
        const float* p0 = &s.v[3 * (size_t)s.t[3 * (size_t)id]];
        const float* p1 = &s.v[3 * (size_t)s.t[3 * (size_t)id + 1]];
        const float* p2 = &s.v[3 * (size_t)s.t[3 * (size_t)id + 2]];
        records = r.v0_id.x == p0[0] && r.v0_id.y == p0[1] && r.v0_id.z == p0[2] && r.e1_mat.x == p1[0] - p0[0] &&
                  r.e1_mat.y == p1[1] - p0[1] && r.e1_mat.z == p1[2] - p0[2] && r.e2.x == p2[0] - p0[0] &&
                  r.e2.y == p2[1] - p0[1] && r.e2.z == p2[2] - p0[2] && mat == (int)s.m[id];
    }
    const std::string mode = argc > 2 ? argv[2] : "";
    if (mode == "shrink" && !a.nodes.empty()) a.nodes[0].lox.x = a.nodes[0].hix.x;
    if (mode == "drop") {
        for (jr::Bvh4Node& n : a.nodes) {
            int* r = &n.refs.x;
            int j = 0;
            while (j < 4 && !(r[j] < 0 && r[j] != jr::kNoChild && ((~r[j]) & 7) > 0)) ++j;
            if (j < 4) {
                r[j] = ~((~r[j]) - 1);  // one triangle fewer in this leaf
                break;
            }
        }
    }
    Checker c{s, a, std::vector<int>(nt, 0)};
    const int need = c.walk(a.root);
    bool cover = true;
    for (uint32_t t = 0; t < nt; ++t) cover = cover && c.seen[t] == 1;
    std::printf("ok=1 same=%d cover=%d records=%d refs=%d empty=%d contain=%d stack=%d need=%d nodes=%zu tris=%zu\n",
                same, cover, records, c.refs, c.empty, c.contain, need + 1 <= jr::kStackSize, need, a.nodes.size(),
                a.tris.size());
    return 0;
}
