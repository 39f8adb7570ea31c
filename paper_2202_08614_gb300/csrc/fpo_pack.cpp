// Host-side validation and breadth-first packing of a union octree (Sec. 4.2):
// the leaves of the union of per-frame octree structures, each a disjoint
// cell of the 2^depth grid at its own depth.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "fpo_internal.h"

namespace fpo {
namespace {

// Interleaves the low 12 bits of x, y, z (x in bit 0): a cell's Morton key at
// the finest level of a depth-M grid.
uint64_t interleave3(uint32_t x, uint32_t y, uint32_t z)
{
    uint64_t k = 0;
    for (int b = 0; b < MAX_DEPTH; ++b) {
        k |= (uint64_t)((x >> b) & 1u) << (3 * b);
        k |= (uint64_t)((y >> b) & 1u) << (3 * b + 1);
        k |= (uint64_t)((z >> b) & 1u) << (3 * b + 2);
    }
    return k;
}

std::string fmt(const char *f, long long a, long long b = 0, long long c = 0)
{
    char buf[256];
    std::snprintf(buf, sizeof buf, f, a, b, c);
    return buf;
}

}  // namespace

int validate_and_pack(const fpo_tree_desc *tree, int n1, int n2, PackedTree *out, std::string *err)
{
    (void)n2;  // n1 == 0 marks a tree without coefficients (latent storage)
    if (!tree) { *err = "tree description is NULL"; return FPO_ERR_INVALID_ARG; }
    const uint32_t n = tree->n_leaves;
    if (tree->max_depth > (uint32_t)MAX_DEPTH) {
        *err = fmt("max_depth %lld exceeds %lld", tree->max_depth, MAX_DEPTH);
        return FPO_ERR_INVALID_ARG;
    }
    if (!(tree->aabb_size > 0.0) || !std::isfinite(tree->aabb_size) ||
        !std::isfinite(tree->aabb_min[0]) || !std::isfinite(tree->aabb_min[1]) ||
        !std::isfinite(tree->aabb_min[2])) {
        *err = "aabb_size must be finite and > 0, aabb_min finite";
        return FPO_ERR_INVALID_ARG;
    }
    if (n > 0 && (!tree->leaf_depth || !tree->leaf_xyz || (!tree->coeffs && n1 > 0))) {
        *err = "leaf_depth, leaf_xyz and coeffs must be non-NULL when n_leaves > 0";
        return FPO_ERR_INVALID_ARG;
    }
    if (n >= LEAF_BIT) { *err = "too many leaves"; return FPO_ERR_INVALID_ARG; }

    // Range checks, then disjointness: a cell at depth d covers the Morton
    // interval [key, key + 8^(M-d)) of the finest level M, so leaves are
    // disjoint iff their sorted intervals do not overlap.
    const int M = (int)tree->max_depth;
    int dmax = 0;
    std::vector<std::pair<uint64_t, uint32_t>> iv(n);
    for (uint32_t j = 0; j < n; ++j) {
        const int d = tree->leaf_depth[j];
        const uint32_t x = tree->leaf_xyz[3 * j], y = tree->leaf_xyz[3 * j + 1],
                       z = tree->leaf_xyz[3 * j + 2];
        if (d > M) {
            *err = fmt("leaf %lld has depth %lld > max_depth %lld", j, d, M);
            return FPO_ERR_BAD_TREE;
        }
        if ((x >> d) || (y >> d) || (z >> d)) {
            *err = fmt("leaf %lld: coordinates outside the 2^%lld grid", j, d);
            return FPO_ERR_BAD_TREE;
        }
        dmax = std::max(dmax, d);
        const int s = M - d;
        iv[j] = {interleave3(x << s, y << s, z << s), j};
    }
    std::sort(iv.begin(), iv.end());
    for (uint32_t i = 0; i + 1 < n; ++i) {
        const uint32_t j = iv[i].second;
        const uint64_t len = 1ull << (3 * (M - (int)tree->leaf_depth[j]));
        if (iv[i].first + len > iv[i + 1].first) {
            *err = fmt("leaves %lld and %lld overlap (duplicate or nested)", j, iv[i + 1].second);
            return FPO_ERR_BAD_TREE;
        }
    }
    if (!out) return FPO_OK;

    // Packing.
    out->nodes.clear();
    out->perm.clear();
    out->depth = dmax;
    if (n == 0) { out->root_kind = ROOT_EMPTY; return FPO_OK; }
    if (dmax == 0) {  // a single leaf covering the whole cube
        out->root_kind = ROOT_LEAF;
        out->perm.push_back(0);
        return FPO_OK;
    }
    out->root_kind = ROOT_NODE;

    // Temporary pointer tree: child >= 0 node, -1 empty, <= -2 leaf -(2 + id).
    struct TNode { int32_t c[8]; };
    std::vector<TNode> tn;
    tn.reserve(n / 4 + 16);
    TNode blank;
    for (int i = 0; i < 8; ++i) blank.c[i] = -1;
    tn.push_back(blank);
    // Insert in Morton order so that siblings are created together.
    for (uint32_t i = 0; i < n; ++i) {
        const uint32_t j = iv[i].second;
        const int d = tree->leaf_depth[j];
        const uint32_t x = tree->leaf_xyz[3 * j], y = tree->leaf_xyz[3 * j + 1],
                       z = tree->leaf_xyz[3 * j + 2];
        int32_t cur = 0;
        for (int l = 0; l < d; ++l) {
            const int sh = d - 1 - l;
            const int c = ((x >> sh) & 1) | (((y >> sh) & 1) << 1) | (((z >> sh) & 1) << 2);
            if (l == d - 1) {
                tn[cur].c[c] = -(2 + (int32_t)j);
            } else {
                if (tn[cur].c[c] == -1) {
                    tn[cur].c[c] = (int32_t)tn.size();
                    tn.push_back(blank);
                }
                cur = tn[cur].c[c];
            }
        }
    }
    // Breadth-first renumbering: nodes in queue order, leaves in slot order.
    out->nodes.resize(tn.size() * 8);
    out->perm.reserve(n);
    std::vector<int32_t> queue;
    queue.reserve(tn.size());
    queue.push_back(0);
    for (size_t qi = 0; qi < queue.size(); ++qi) {
        const TNode &t = tn[queue[qi]];
        for (int c = 0; c < 8; ++c) {
            uint32_t slot = 0;
            if (t.c[c] >= 0) {
                slot = (uint32_t)queue.size();
                queue.push_back(t.c[c]);
            } else if (t.c[c] <= -2) {
                slot = LEAF_BIT | (uint32_t)out->perm.size();
                out->perm.push_back((uint32_t)(-(t.c[c] + 2)));
            }
            out->nodes[qi * 8 + c] = slot;
        }
    }
    return FPO_OK;
}

namespace {

// Encodes |x| into a sign-less minifloat with E exponent bits, M mantissa
// bits and the given bias, rounding to nearest even; returns the code or -1
// when the rounded value exceeds the largest finite value max_val.
long minifloat_abs(double a, int E, int M, int bias, double max_val)
{
    if (a == 0.0) return 0;
    int e2;
    std::frexp(a, &e2);           // a = f * 2^e2, f in [0.5, 1)
    int ue = e2 - 1;              // a = 1.x * 2^ue
    const int emin = 1 - bias;    // smallest normal exponent
    long code;
    if (ue < emin) {              // subnormal: units of 2^(emin - M)
        const double q = std::nearbyint(std::ldexp(a, M - emin));
        code = (long)q;           // q == 2^M rolls into the smallest normal
    } else {
        double q = std::nearbyint(std::ldexp(a, M - ue));  // in [2^M, 2^(M+1)]
        if (q >= std::ldexp(1.0, M + 1)) {
            q *= 0.5;
            ++ue;
        }
        code = ((long)(ue + bias) << M) | ((long)q - (1L << M));
    }
    // decode to compare against the largest finite value
    const long ef = code >> M, mf = code & ((1L << M) - 1);
    const double v = ef == 0 ? std::ldexp((double)mf, emin - M)
                             : std::ldexp(1.0 + std::ldexp((double)mf, -M), (int)ef - bias);
    if (v > max_val || ef >= (1L << E)) return -1;
    return code;
}

}  // namespace

uint16_t encode_bf16(float x)
{
    if (std::isnan(x)) return 0x7FC0;
    const uint16_t s = std::signbit(x) ? 0x8000 : 0;
    const long c = minifloat_abs(std::fabs((double)x), 8, 7, 127, 3.3895313892515355e38);
    return (uint16_t)(s | (c < 0 ? 0x7F80 : c));  // overflow -> infinity
}

uint16_t encode_f16(float x)
{
    if (std::isnan(x)) return 0x7E00;
    const uint16_t s = std::signbit(x) ? 0x8000 : 0;
    const long c = minifloat_abs(std::fabs((double)x), 5, 10, 15, 65504.0);
    return (uint16_t)(s | (c < 0 ? 0x7C00 : c));  // overflow -> infinity
}

uint8_t encode_e4m3(float x)
{
    if (std::isnan(x)) return 0x7F;
    const uint8_t s = std::signbit(x) ? 0x80 : 0;
    long c = minifloat_abs(std::fabs((double)x), 4, 3, 7, 448.0);
    if (c < 0 || c > 0x7E) c = 0x7E;  // saturate at 448 (0x7F is NaN)
    return (uint8_t)(s | c);
}

}  // namespace fpo
