// Union of per-frame octree structures (Sec. 4.2): the unified octree whose
// leaves are at least as deep as every frame's, with each frame's values
// copied into the leaves its own (coarser) leaf was divided into.
#include <cstring>
#include <string>
#include <vector>

#include "fpo_internal.h"

namespace fpo {
namespace {

struct UNode {
    int32_t child[8];
    int32_t mark;  // head of this cell's (frame, value) list, -1 if none
};
struct Mark {
    uint32_t frame, leaf;
    int32_t next;
};

struct Builder {
    std::vector<UNode> nodes;
    std::vector<Mark> marks;
    uint32_t n_frames = 0;
    const fpo_frame_tree *frames = nullptr;
    // output
    uint64_t n_out = 0;
    uint32_t cap = 0;
    uint8_t *depth_out = nullptr;
    uint32_t *xyz_out = nullptr;
    float *values_out = nullptr;

    int32_t new_node()
    {
        UNode u;
        for (int i = 0; i < 8; ++i) u.child[i] = -1;
        u.mark = -1;
        nodes.push_back(u);
        return (int32_t)nodes.size() - 1;
    }

    void emit(int d, uint32_t x, uint32_t y, uint32_t z, const int32_t *cover)
    {
        const uint64_t u = n_out++;
        if (u >= cap) return;  // counting pass
        depth_out[u] = (uint8_t)d;
        xyz_out[3 * u] = x;
        xyz_out[3 * u + 1] = y;
        xyz_out[3 * u + 2] = z;
        for (uint32_t f = 0; f < n_frames; ++f) {
            float *dst = values_out + ((size_t)f * cap + u) * 28;
            if (cover[f] >= 0)
                std::memcpy(dst, frames[f].values + (size_t)cover[f] * 28, 28 * sizeof(float));
            else
                std::memset(dst, 0, 28 * sizeof(float));
        }
    }

    // cover[f]: the frame-f leaf holding this cell (the cell or an ancestor), or -1
    void walk(int32_t n, int d, uint32_t x, uint32_t y, uint32_t z, std::vector<int32_t> &cover)
    {
        std::vector<int32_t> saved;
        for (int32_t m = nodes[n].mark; m >= 0; m = marks[m].next) {
            saved.push_back((int32_t)marks[m].frame);
            saved.push_back(cover[marks[m].frame]);
            cover[marks[m].frame] = (int32_t)marks[m].leaf;
        }
        bool split = false;
        for (int c = 0; c < 8; ++c) split |= nodes[n].child[c] >= 0;
        if (!split) {
            emit(d, x, y, z, cover.data());
        } else {
            bool covered = false;
            for (uint32_t f = 0; f < n_frames; ++f) covered |= cover[f] >= 0;
            for (int c = 0; c < 8; ++c) {
                const uint32_t cx = 2 * x + (c & 1), cy = 2 * y + ((c >> 1) & 1), cz = 2 * z + ((c >> 2) & 1);
                if (nodes[n].child[c] >= 0)
                    walk(nodes[n].child[c], d + 1, cx, cy, cz, cover);
                else if (covered)  // a divided leaf: its value is copied into the new leaves
                    emit(d + 1, cx, cy, cz, cover.data());
            }
        }
        for (size_t i = saved.size(); i > 0; i -= 2) cover[saved[i - 2]] = saved[i - 1];
    }
};

}  // namespace
}  // namespace fpo

using namespace fpo;

extern "C" int fpo_union_trees(uint32_t n_frames, const fpo_frame_tree *frames, uint32_t max_depth,
                               uint32_t *n_union, uint8_t *union_depth, uint32_t *union_xyz,
                               float *union_values, uint32_t capacity)
{
    if (!n_union || (n_frames > 0 && !frames)) return set_last_error(FPO_ERR_INVALID_ARG, "NULL argument");
    if (capacity > 0 && (!union_depth || !union_xyz || !union_values))
        return set_last_error(FPO_ERR_INVALID_ARG, "output arrays are NULL");
    *n_union = 0;
    Builder b;
    b.n_frames = n_frames;
    b.frames = frames;
    b.new_node();
    for (uint32_t f = 0; f < n_frames; ++f) {
        const fpo_frame_tree &fr = frames[f];
        if (fr.n_leaves > 0 && !fr.values)
            return set_last_error(FPO_ERR_INVALID_ARG, "frame values are NULL");
        // each frame is a valid octree on its own (disjoint leaves in range)
        fpo_tree_desc desc{};
        desc.n_leaves = fr.n_leaves;
        desc.max_depth = max_depth;
        desc.leaf_depth = fr.leaf_depth;
        desc.leaf_xyz = fr.leaf_xyz;
        desc.coeffs = fr.values;
        desc.aabb_size = 1.0;
        std::string err;
        const int st = validate_and_pack(&desc, 1, 1, nullptr, &err);
        if (st != FPO_OK) return set_last_error(st, ("frame " + std::to_string(f) + ": " + err).c_str());
        for (uint32_t j = 0; j < fr.n_leaves; ++j) {
            const int d = fr.leaf_depth[j];
            const uint32_t x = fr.leaf_xyz[3 * j], y = fr.leaf_xyz[3 * j + 1], z = fr.leaf_xyz[3 * j + 2];
            int32_t cur = 0;
            for (int l = 0; l < d; ++l) {
                const int sh = d - 1 - l;
                const int c = ((x >> sh) & 1) | (((y >> sh) & 1) << 1) | (((z >> sh) & 1) << 2);
                if (b.nodes[cur].child[c] < 0) {
                    const int32_t nn = b.new_node();
                    b.nodes[cur].child[c] = nn;
                }
                cur = b.nodes[cur].child[c];
            }
            b.marks.push_back({f, j, b.nodes[cur].mark});
            b.nodes[cur].mark = (int32_t)b.marks.size() - 1;
        }
    }
    b.cap = capacity;
    b.depth_out = union_depth;
    b.xyz_out = union_xyz;
    b.values_out = union_values;
    std::vector<int32_t> cover(n_frames, -1);
    bool any = false;
    for (uint32_t f = 0; f < n_frames; ++f) any |= frames[f].n_leaves > 0;
    if (any) b.walk(0, 0, 0, 0, 0, cover);
    if (b.n_out >= LEAF_BIT) return set_last_error(FPO_ERR_INVALID_ARG, "union has too many leaves");
    *n_union = (uint32_t)b.n_out;
    if (capacity > 0 && b.n_out > capacity)
        return set_last_error(FPO_ERR_INVALID_ARG, "capacity is smaller than the union");
    return FPO_OK;
}
