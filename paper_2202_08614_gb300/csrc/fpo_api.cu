// The C ABI of the FPO renderer (include/fpo.h): context, tree upload,
// render dispatch and device status.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "fpo_internal.h"

using namespace fpo;

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(e == cudaErrorMemoryAllocation ? FPO_ERR_OOM : FPO_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

template <class T>
void dfree(T *&p)
{
    if (p) cudaFree((void *)p);
    p = nullptr;
}

// Launch shapes of the frame pipeline (fpo_render_frames).  The traversal of
// frame k and the IDFT pass of frame k + 1 share every SM: two 384-thread
// traversal CTAs (64 registers a thread) leave a quarter of the register file
// to the IDFT pass (materialise_pipeline_shape: one 128-thread CTA of the
// thread-per-leaf form, or two 256-thread CTAs of the warp-cooperative form),
// whose stage rings are capped so that all CTAs' shared memory fits one
// carveout.
#ifndef FPO_PIPE_TRAV_THREADS
#define FPO_PIPE_TRAV_THREADS 384
#endif
#ifndef FPO_PIPE_TRAV_CTAS
#define FPO_PIPE_TRAV_CTAS 2
#endif
#ifndef FPO_PIPE_MAT_CTAS
#define FPO_PIPE_MAT_CTAS 0  // IDFT-pass CTAs per SM in the pipeline (0: materialise_pipeline_shape's choice)
#endif
#ifndef FPO_PIPE_DEPTH
// Tables (and traversal streams) in flight in fpo_render_frames.  Measured
// (FP32 / BF16 1080p frames, ms): depth 2 0.675 / 0.516, 3 0.656 / 0.486,
// 4 0.639 / 0.457, 5 0.653 / 0.480, 6 0.648 / 0.465, 8 0.649 / 0.469.
#define FPO_PIPE_DEPTH 4
#endif
constexpr int PIPE_MAX = 8;
static_assert(FPO_PIPE_DEPTH >= 2 && FPO_PIPE_DEPTH <= PIPE_MAX, "pipeline depth");
#ifndef FPO_PIPE_SLOT_STREAMS
#define FPO_PIPE_SLOT_STREAMS 1  // each pipeline slot's traversals on its own stream (0: all on the caller's)
#endif
#ifndef FPO_PIPE_MAT_SMEM_KB
#define FPO_PIPE_MAT_SMEM_KB 88
#endif
constexpr int PIPE_TRAV_THREADS = FPO_PIPE_TRAV_THREADS;
constexpr int PIPE_TRAV_CTAS = FPO_PIPE_TRAV_CTAS;
constexpr int PIPE_MAT_SMEM_BUDGET = FPO_PIPE_MAT_SMEM_KB * 1024;  // bytes of coefficient records in flight per SM
constexpr int PIPE_STATIC_SMEM = 512;            // allowance for each kernel's static shared memory
constexpr int SMEM_CONFIGS_KB[] = {0, 8, 16, 32, 64, 100, 132, 164, 196, 228};  // per SM, sm_100 family
// Top-level nodes staged in shared memory per traversal CTA (32 B each); 0
// with the kernels' default FPO_NODE_SMEM 0, which reads every node slot
// from global memory.
#ifndef FPO_SMEM_NODES
#define FPO_SMEM_NODES 0
#endif
constexpr uint32_t SMEM_NODE_BUDGET = FPO_SMEM_NODES;
constexpr int DEFAULT_TRAVERSE_THREADS = 256;
constexpr uint32_t DEFAULT_REFILL_MIN = 32;
constexpr uint32_t DEFAULT_INNER_STEPS = 0xffffffffu;  // a lane runs its ray to the end

}  // namespace

struct fpo_ctx {
    fpo_config cfg{};
    int sm_count = 0;
    // [0] status bits; [1], [2] tile counter and finished warps of a traversal;
    // [5], [6] the same for the odd frames of fpo_render_frames, whose
    // traversals run on a second stream and may overlap the even ones
    uint32_t *d_status = nullptr;
    // tree
    bool has_tree = false;
    uint32_t n_leaves = 0, n_nodes = 0, root_kind = ROOT_EMPTY, n_smem_nodes = 0;
    int depth = 0;
    uint32_t max_depth = 0;
    double aabb_min[3] = {0, 0, 0}, aabb_size = 1.0;
    uint32_t *d_nodes = nullptr;
    uint32_t *d_perm = nullptr;
    void *d_sig = nullptr;    // density records (storage precision)
    void *d_z = nullptr;      // SH records (storage precision)
    float *d_scale = nullptr; // FP8: per-leaf scale, padded to a multiple of 4 leaves
    uint16_t *d_latents = nullptr;  // LATENT: FP16 [n_leaves][32], internal leaf order
    uint16_t *d_dec_w = nullptr;    // LATENT: w1 | w2 | w3 (BF16 bits)
    float *d_dec_b = nullptr;       // LATENT: b1 | b2 | b3
    bool has_latents = false;
    float *d_table = nullptr;
    size_t table_leaves = 0;
    // frame pipeline (fpo_render_frames): second table, aux stream, events
    bool half_table = false;  // the per-frame table holds FP16 (64 B per leaf)
    bool table_ok = false;    // d_table holds the IDFT pass of table_t for the current coefficients
    double table_t = 0.0;
    // slot b of the pipeline: frames b, b + depth, ... (slot 0: d_table, the caller's stream)
    float *d_ptable[PIPE_MAX] = {};       // slots 1.. : their tables
    size_t ptable_leaves[PIPE_MAX] = {};
    cudaStream_t aux = nullptr;           // IDFT passes / decodes
    cudaStream_t trav[PIPE_MAX] = {};     // slots 1.. : their traversal streams
    cudaEvent_t ev_entry = nullptr, ev_mat[PIPE_MAX] = {}, ev_trav[PIPE_MAX] = {};

    void free_tree()
    {
        dfree(d_nodes);
        dfree(d_perm);
        dfree(d_sig);
        dfree(d_z);
        dfree(d_scale);
        dfree(d_latents);
        dfree(d_dec_w);
        dfree(d_dec_b);
        has_latents = false;
        dfree(d_table);
        table_leaves = 0;
        table_ok = false;
        for (int b = 1; b < PIPE_MAX; ++b) {
            dfree(d_ptable[b]);
            ptable_leaves[b] = 0;
        }
        has_tree = false;
    }
};

namespace fpo {

// Bytes of one leaf's row of the per-frame table.
static size_t table_row_bytes(const fpo_ctx *c) { return c->half_table ? TABLE_STRIDE * 2 : TABLE_STRIDE * 4; }
// Bytes of a per-frame table: rows rounded up to a multiple of 8 leaves, so
// that a prefetch of the aligned 512-byte group of rows holding any leaf
// stays inside the allocation.
static size_t table_alloc_bytes(const fpo_ctx *c) { return (((size_t)c->n_leaves + 7) & ~(size_t)7) * table_row_bytes(c); }

CtxView ctx_view(const fpo_ctx *c)
{
    CtxView v{};
    v.device = c->cfg.device;
    v.sm_count = c->sm_count;
    v.n1 = c->cfg.n1;
    v.n2 = c->cfg.n2;
    v.period_T = c->cfg.period_T;
    v.traverse_threads = c->cfg.traverse_threads;
    v.refill_min = c->cfg.refill_min;
    v.inner_steps = c->cfg.inner_steps;
    v.max_steps = c->cfg.max_steps;
    v.d_status = c->d_status;
    v.half_table = c->half_table;
    v.has_tree = c->has_tree;
    v.n_leaves = c->n_leaves;
    v.n_nodes = c->n_nodes;
    v.root_kind = c->root_kind;
    v.n_smem_nodes = c->n_smem_nodes;
    v.depth = c->depth;
    for (int k = 0; k < 3; ++k) v.aabb_min[k] = c->aabb_min[k];
    v.aabb_size = c->aabb_size;
    v.d_nodes = c->d_nodes;
    v.d_perm = c->d_perm;
    v.storage = c->cfg.storage;
    v.d_sig = c->d_sig;
    v.d_z = c->d_z;
    v.d_scale = c->d_scale;
    return v;
}

int set_last_error(int code, const char *msg) { return fail(code, "%s", msg); }

}  // namespace fpo

extern "C" {

const char *fpo_last_error(void) { return g_err.c_str(); }

int fpo_version(void) { return 102; }

int fpo_create(fpo_ctx **out, const fpo_config *cfg)
{
    if (!out) return fail(FPO_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!cfg) return fail(FPO_ERR_INVALID_ARG, "cfg is NULL");
    if (cfg->n1 < 1 || cfg->n1 > 32) return fail(FPO_ERR_INVALID_ARG, "n1 must be in [1, 32]");
    if (cfg->n2 < 1 || cfg->n2 > 16) return fail(FPO_ERR_INVALID_ARG, "n2 must be in [1, 16]");
    if (cfg->sh_degree != 2) return fail(FPO_ERR_UNSUPPORTED, "only sh_degree 2 is supported");
    if (!(cfg->period_T > 0.0) || !std::isfinite(cfg->period_T))
        return fail(FPO_ERR_INVALID_ARG, "period_T must be finite and > 0");
    if (cfg->storage < FPO_STORAGE_F32 || cfg->storage > FPO_STORAGE_LATENT)
        return fail(FPO_ERR_INVALID_ARG, "unknown storage %d", cfg->storage);
    if (cfg->idft_mode < FPO_IDFT_AUTO || cfg->idft_mode > FPO_IDFT_MATERIALISE)
        return fail(FPO_ERR_INVALID_ARG, "unknown idft_mode %d", cfg->idft_mode);
    if (cfg->traverse_threads != 0 && cfg->traverse_threads != 128 && cfg->traverse_threads != 256)
        return fail(FPO_ERR_INVALID_ARG, "traverse_threads must be 0, 128 or 256");
    if (cfg->refill_min < 0 || cfg->refill_min > 32)
        return fail(FPO_ERR_INVALID_ARG, "refill_min must be in [0, 32]");
    if (cfg->inner_steps < 0) return fail(FPO_ERR_INVALID_ARG, "inner_steps must be >= 0");
    if (cfg->max_steps < 0) return fail(FPO_ERR_INVALID_ARG, "max_steps must be >= 0");
    if (cfg->table_precision < FPO_TABLE_AUTO || cfg->table_precision > FPO_TABLE_F16)
        return fail(FPO_ERR_INVALID_ARG, "table_precision must be FPO_TABLE_AUTO, _F32 or _F16");
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (cfg->device < 0 || cfg->device >= ndev)
        return fail(FPO_ERR_INVALID_ARG, "device %d out of range (%d devices)", cfg->device, ndev);
    DeviceGuard g(cfg->device);
    if (!g.ok) return fail(FPO_ERR_CUDA, "cudaSetDevice(%d) failed", cfg->device);
    fpo_ctx *c = new (std::nothrow) fpo_ctx;
    if (!c) return fail(FPO_ERR_OOM, "host allocation failed");
    c->cfg = *cfg;
    c->half_table = cfg->table_precision == FPO_TABLE_F16 ||
                    (cfg->table_precision == FPO_TABLE_AUTO && cfg->storage != FPO_STORAGE_F32);
    e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, cfg->device);
    if (e != cudaSuccess) { delete c; return cuda_fail(e, "cudaDeviceGetAttribute"); }
    e = cudaMalloc((void **)&c->d_status, 32 * sizeof(uint32_t));
    if (e != cudaSuccess) { delete c; return cuda_fail(e, "cudaMalloc(status)"); }
    e = cudaMemset(c->d_status, 0, 32 * sizeof(uint32_t));
    if (e != cudaSuccess) { cudaFree(c->d_status); delete c; return cuda_fail(e, "cudaMemset"); }
    *out = c;
    g_err.clear();
    return FPO_OK;
}

int fpo_validate_tree(const fpo_tree_desc *tree, const fpo_config *cfg)
{
    if (!cfg) return fail(FPO_ERR_INVALID_ARG, "cfg is NULL");
    std::string err;
    int st = validate_and_pack(tree, cfg->n1, cfg->n2, nullptr, &err);
    if (st != FPO_OK) return fail(st, "%s", err.c_str());
    return FPO_OK;
}

int fpo_upload_tree(fpo_ctx *ctx, const fpo_tree_desc *tree)
{
    if (!ctx) return fail(FPO_ERR_INVALID_ARG, "ctx is NULL");
    PackedTree pk;
    std::string err;
    const bool latent = ctx->cfg.storage == FPO_STORAGE_LATENT;
    int st = validate_and_pack(tree, latent ? 0 : ctx->cfg.n1, ctx->cfg.n2, &pk, &err);
    if (st != FPO_OK) return fail(st, "%s", err.c_str());
    DeviceGuard g(ctx->cfg.device);
    if (!g.ok) return fail(FPO_ERR_CUDA, "cudaSetDevice failed");
    ctx->free_tree();

    const int n1 = ctx->cfg.n1, n2 = ctx->cfg.n2, nc = n1 + 27 * n2;
    const int storage = ctx->cfg.storage;
    const RecordLayout L = record_layout(latent ? FPO_STORAGE_F32 : storage, n1, n2);
    const size_t n = latent ? 0 : tree->n_leaves;  // latent storage keeps no coefficient records
    // Reorder the coefficients into breadth-first leaf order, split into the
    // density and the SH record arrays (zero padded), encoded in the storage
    // precision; FP8 codes hold coefficient / scale with a per-leaf scale
    // max|k| / 448 (448 = the largest E4M3 value).
    std::vector<uint8_t> sig(n * L.sig_bytes(), 0), zc(n * L.z_bytes(), 0);
    std::vector<float> scale(L.scaled ? (n + 3) / 4 * 4 : 0, 0.0f);
    auto put = [&](uint8_t *rec, int j, float v) {
        switch (storage) {
        case FPO_STORAGE_BF16: { const uint16_t c = encode_bf16(v); std::memcpy(rec + 2 * j, &c, 2); break; }
        case FPO_STORAGE_F16: { const uint16_t c = encode_f16(v); std::memcpy(rec + 2 * j, &c, 2); break; }
        case FPO_STORAGE_FP8_E4M3: rec[j] = encode_e4m3(v); break;
        default: std::memcpy(rec + 4 * j, &v, 4);
        }
    };
    for (size_t i = 0; i < n; ++i) {
        const float *src = tree->coeffs + (size_t)pk.perm[i] * nc;
        float sc = 1.0f;
        if (L.scaled) {
            float mx = 0.0f;
            for (int j = 0; j < nc; ++j) mx = std::fmax(mx, std::fabs(src[j]));
            sc = mx > 0.0f ? mx / 448.0f : 1.0f;
            scale[i] = sc;
        }
        uint8_t *rs = &sig[i * L.sig_bytes()];
        uint8_t *rz = &zc[i * L.z_bytes()];
        for (int j = 0; j < n1; ++j) put(rs, j, L.scaled ? src[j] / sc : src[j]);
        for (int j = 0; j < 27 * n2; ++j) put(rz, j, L.scaled ? src[n1 + j] / sc : src[n1 + j]);
    }
    const size_t n_nodes = pk.nodes.size() / 8;
    cudaError_t e = cudaSuccess;
    auto up = [&](void **dst, const void *src, size_t bytes, const char *what) -> int {
        if (bytes == 0) return FPO_OK;
        e = cudaMalloc(dst, bytes);
        if (e != cudaSuccess) return cuda_fail(e, what);
        e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, what);
        return FPO_OK;
    };
    if ((st = up((void **)&ctx->d_nodes, pk.nodes.data(), pk.nodes.size() * 4, "nodes")) ||
        (st = up((void **)&ctx->d_perm, pk.perm.data(), pk.perm.size() * 4, "perm")) ||
        (st = up((void **)&ctx->d_sig, sig.data(), sig.size(), "sigma records")) ||
        (st = up((void **)&ctx->d_z, zc.data(), zc.size(), "SH records")) ||
        (st = up((void **)&ctx->d_scale, scale.data(), scale.size() * 4, "FP8 scales"))) {
        ctx->free_tree();
        return st;
    }
    ctx->n_leaves = tree->n_leaves;
    ctx->n_nodes = (uint32_t)n_nodes;
    ctx->root_kind = pk.root_kind;
    ctx->depth = pk.depth;
    ctx->max_depth = tree->max_depth;
    ctx->n_smem_nodes = (uint32_t)(n_nodes < SMEM_NODE_BUDGET ? n_nodes : SMEM_NODE_BUDGET);
    for (int k = 0; k < 3; ++k) ctx->aabb_min[k] = tree->aabb_min[k];
    ctx->aabb_size = tree->aabb_size;
    ctx->has_tree = true;
    g_err.clear();
    return FPO_OK;
}

int fpo_tree_info_get(const fpo_ctx *ctx, fpo_tree_info *out)
{
    if (!ctx || !out) return fail(FPO_ERR_INVALID_ARG, "NULL argument");
    if (!ctx->has_tree) return fail(FPO_ERR_NO_TREE, "no tree uploaded");
    out->n_leaves = ctx->n_leaves;
    out->n_nodes = ctx->n_nodes;
    out->max_depth = ctx->max_depth;
    out->n_smem_nodes = ctx->n_smem_nodes;
    out->node_bytes = (uint64_t)ctx->n_nodes * 32;
    if (ctx->cfg.storage == FPO_STORAGE_LATENT) {
        out->leaf_record_bytes = 64;  // one FP16 latent of 32 values (the decoder is shared)
    } else {
        const RecordLayout L = record_layout(ctx->cfg.storage, ctx->cfg.n1, ctx->cfg.n2);
        out->leaf_record_bytes = (uint64_t)(L.sig_bytes() + L.z_bytes() + (L.scaled ? 4 : 0));
    }
    out->leaf_bytes = out->leaf_record_bytes * ctx->n_leaves;
    out->table_bytes = (uint64_t)ctx->table_leaves * table_row_bytes(ctx);
    return FPO_OK;
}

}  // extern "C"

namespace fpo {

int check_rays(const fpo_rays *r, uint64_t *n_rays)
{
    if (r->mode == FPO_RAYS_CAMERA) {
        const double fov = r->fov_y_deg;
        if (!(fov > 0.0 && fov < 180.0)) return fail(FPO_ERR_INVALID_ARG, "fov_y_deg must be in (0, 180)");
        double f[3], c[3];
        for (int k = 0; k < 3; ++k) f[k] = r->target[k] - r->eye[k];
        c[0] = f[1] * r->up[2] - f[2] * r->up[1];
        c[1] = f[2] * r->up[0] - f[0] * r->up[2];
        c[2] = f[0] * r->up[1] - f[1] * r->up[0];
        const double fl = f[0] * f[0] + f[1] * f[1] + f[2] * f[2];
        const double cl = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
        if (!(fl > 0.0) || !(cl > 0.0) || !std::isfinite(fl) || !std::isfinite(cl))
            return fail(FPO_ERR_INVALID_ARG, "degenerate camera (eye == target or up parallel to the view)");
        if (!std::isfinite(r->t)) return fail(FPO_ERR_INVALID_ARG, "t must be finite");
        *n_rays = (uint64_t)r->width * r->height;
    } else if (r->mode == FPO_RAYS_EXPLICIT) {
        if (r->n > 0 && (!r->o || !r->d)) return fail(FPO_ERR_INVALID_ARG, "o and d must be non-NULL");
        if (!r->t_per_ray && !std::isfinite(r->t)) return fail(FPO_ERR_INVALID_ARG, "t must be finite");
        *n_rays = r->n;
    } else {
        return fail(FPO_ERR_INVALID_ARG, "unknown ray mode %d", r->mode);
    }
    if (*n_rays >= (1ull << 31)) return fail(FPO_ERR_INVALID_ARG, "too many rays");
    return FPO_OK;
}

int check_render_opts(const fpo_ctx *ctx, const fpo_frame_opts *opts, uint64_t n_rays, const float *out_rgb)
{
    if (n_rays > 0 && !out_rgb) return fail(FPO_ERR_INVALID_ARG, "out_rgb is NULL");
    const uint32_t fl = opts->flags;
    if ((fl & FPO_FLAG_RECORD_VISITS) && (!opts->visit_count || (opts->visit_cap && !opts->visit_log)))
        return fail(FPO_ERR_INVALID_ARG, "RECORD_VISITS needs visit_count (and visit_log if visit_cap > 0)");
    if ((fl & FPO_FLAG_OUT_T) && !opts->out_T) return fail(FPO_ERR_INVALID_ARG, "OUT_T needs out_T");
    if ((fl & FPO_FLAG_STATS) && !opts->stats) return fail(FPO_ERR_INVALID_ARG, "STATS needs stats");
    if ((fl & FPO_FLAG_MARK_LEAVES) && !opts->leaf_mark && ctx->n_leaves)
        return fail(FPO_ERR_INVALID_ARG, "MARK_LEAVES needs leaf_mark");
    if (!(opts->stop_T >= 0.0f)) return fail(FPO_ERR_INVALID_ARG, "stop_T must be >= 0");
    return FPO_OK;
}

// Kernel parameters of one render (or adjoint) call from the context, rays
// and options.
TraverseParams traverse_params(const fpo_ctx *ctx, const fpo_rays *rays, const fpo_frame_opts *opts,
                               float *out_rgb, uint64_t n_rays)
{
    const uint32_t fl = opts->flags;
    TraverseParams p{};
    p.fr.mode = rays->mode;
    p.fr.width = rays->width;
    p.fr.height = rays->height;
    p.fr.n_rays = (uint32_t)n_rays;
    for (int k = 0; k < 3; ++k) {
        p.fr.eye[k] = rays->eye[k];
        p.fr.target[k] = rays->target[k];
        p.fr.up[k] = rays->up[k];
    }
    p.fr.fov_y_deg = rays->fov_y_deg;
    p.fr.t = rays->t;
    p.fr.period_T = ctx->cfg.period_T;
    p.fr.ro = rays->o;
    p.fr.rd = rays->d;
    p.fr.rt = rays->t_per_ray;
    p.nodes = ctx->d_nodes;
    p.root_kind = ctx->root_kind;
    p.depth = ctx->depth;
    p.n_smem_nodes = ctx->n_smem_nodes;
    p.grid_scale64 = (double)(1u << ctx->depth) / ctx->aabb_size;
    p.grid_scale = (float)p.grid_scale64;
    for (int k = 0; k < 3; ++k) {
        p.amin64[k] = ctx->aabb_min[k];
        p.amin[k] = (float)ctx->aabb_min[k];
    }
    p.table = reinterpret_cast<const float4 *>(ctx->d_table);
    p.sig = reinterpret_cast<const float4 *>(ctx->d_sig);
    p.zc = static_cast<const float *>(ctx->d_z);
    p.n1 = ctx->cfg.n1;
    p.n2 = ctx->cfg.n2;
    p.sig_stride4 = sig_stride(ctx->cfg.n1) / 4;
    p.z_stride = z_stride(ctx->cfg.n2);
    for (int k = 0; k < 3; ++k) p.bg[k] = opts->bg[k];
    p.stop_T = opts->stop_T;
    p.flags = fl;
    p.out_rgb = out_rgb;
    p.out_T = opts->out_T;
    p.visit_log = opts->visit_log;
    p.visit_cap = opts->visit_cap;
    p.visit_count = opts->visit_count;
    p.leaf_mark = opts->leaf_mark;
    p.perm = ctx->d_perm;
    p.status = ctx->d_status;
    p.tiles = ctx->d_status + 1;
    p.half_table = ctx->half_table;
    if (rays->mode == FPO_RAYS_CAMERA) {
        p.tiles_x = (rays->width + TILE_W - 1) / TILE_W;
        const uint32_t tiles_y = (rays->height + TILE_H - 1) / TILE_H;
        p.n_tiles = p.tiles_x * tiles_y;
    } else {
        p.tiles_x = 0;
        p.n_tiles = (uint32_t)((n_rays + 31) / 32);
    }
    p.max_steps = ctx->cfg.max_steps > 0 ? (uint32_t)ctx->cfg.max_steps : 3u * (1u << ctx->depth) + 16u;
    p.block_threads = ctx->cfg.traverse_threads ? ctx->cfg.traverse_threads : DEFAULT_TRAVERSE_THREADS;
    p.refill_min = ctx->cfg.refill_min ? (uint32_t)ctx->cfg.refill_min : DEFAULT_REFILL_MIN;
    p.inner_steps = ctx->cfg.inner_steps ? (uint32_t)ctx->cfg.inner_steps : DEFAULT_INNER_STEPS;
    p.stats = reinterpret_cast<unsigned long long *>(opts->stats);
    return p;
}

// The per-frame table for time t into `table` on stream s: the tensor-core
// decoder for LATENT storage, else the bulk-copy IDFT pass over the stored
// coefficients (at most max_ctas_per_sm CTAs per SM when > 0).
// With pipe_stages > 0 the pass takes the frame-pipeline shape with that many
// stages (materialise_pipeline_shape), co-scheduled with the traversal.
int launch_table_pass(const fpo_ctx *ctx, double t, float *table, int max_ctas_per_sm, void *stream,
                      int pipe_stages, int carveout, bool test_timeout)
{
    const cudaStream_t s = (cudaStream_t)stream;
    if (ctx->cfg.storage == FPO_STORAGE_LATENT) {
        LatentParams lp{};
        lp.latents = ctx->d_latents;
        lp.w1 = ctx->d_dec_w;
        lp.w2 = ctx->d_dec_w + 64 * 32;
        lp.w3 = ctx->d_dec_w + 64 * 32 + 64 * 64;
        lp.b1 = ctx->d_dec_b;
        lp.b2 = ctx->d_dec_b + 64;
        lp.b3 = ctx->d_dec_b + 128;
        lp.n1 = ctx->cfg.n1;
        lp.n2 = ctx->cfg.n2;
        lp.t = t;
        lp.period_T = ctx->cfg.period_T;
        lp.n_leaves = ctx->n_leaves;
        lp.table = table;
        lp.half_table = ctx->half_table;
        lp.status = ctx->d_status;
        lp.test_timeout = test_timeout;
        lp.pipeline = pipe_stages > 0;
        lp.carveout = carveout;
        return launch_latent_table(lp, ctx->sm_count, s);
    }
    MaterialiseParams mp{};
    const RecordLayout L = record_layout(ctx->cfg.storage, ctx->cfg.n1, ctx->cfg.n2);
    mp.sig = ctx->d_sig;
    mp.zc = ctx->d_z;
    mp.scale = ctx->d_scale;
    mp.table = table;
    mp.n_leaves = ctx->n_leaves;
    mp.storage = ctx->cfg.storage;
    mp.n1 = ctx->cfg.n1;
    mp.n2 = ctx->cfg.n2;
    mp.sig_stride = L.sig_elems;
    mp.z_stride = L.z_elems;
    mp.stages = pipe_stages > 0 ? pipe_stages : materialise_stages(ctx->cfg.storage, ctx->cfg.n1, ctx->cfg.n2);
    mp.pipeline = pipe_stages > 0;
    mp.max_ctas_per_sm = max_ctas_per_sm;
    mp.carveout = carveout;
    mp.half_table = ctx->half_table;
    mp.t = t;
    mp.period_T = ctx->cfg.period_T;
    mp.status = ctx->d_status;
    mp.test_timeout = test_timeout;
    return launch_materialise(mp, ctx->sm_count, s);
}

}  // namespace fpo

extern "C" {

int fpo_render(fpo_ctx *ctx, const fpo_rays *rays, const fpo_frame_opts *opts, float *out_rgb,
               void *cuda_stream)
{
    if (!ctx || !rays || !opts) return fail(FPO_ERR_INVALID_ARG, "NULL argument");
    if (!ctx->has_tree) return fail(FPO_ERR_NO_TREE, "render before fpo_upload_tree");
    uint64_t n_rays = 0;
    int st = check_rays(rays, &n_rays);
    if (st != FPO_OK) return st;
    if ((st = check_render_opts(ctx, opts, n_rays, out_rgb)) != FPO_OK) return st;
    const uint32_t fl = opts->flags;
    const bool per_ray_t = rays->mode == FPO_RAYS_EXPLICIT && rays->t_per_ray;
    int mode = ctx->cfg.idft_mode;
    if (mode == FPO_IDFT_AUTO) mode = per_ray_t ? FPO_IDFT_FUSED : FPO_IDFT_MATERIALISE;
    if (mode == FPO_IDFT_MATERIALISE && per_ray_t)
        return fail(FPO_ERR_INVALID_ARG, "per-ray times need the FUSED IDFT mode");
    const bool mat = mode == FPO_IDFT_MATERIALISE && ctx->n_leaves > 0;
    if (!mat && ctx->n_leaves > 0 && ctx->cfg.storage != FPO_STORAGE_F32)
        return fail(FPO_ERR_UNSUPPORTED, "the fused IDFT reads FP32 records only; use the table mode");
    if (mat && ctx->cfg.storage == FPO_STORAGE_LATENT && !ctx->has_latents)
        return fail(FPO_ERR_INVALID_ARG, "LATENT storage: call fpo_set_latents before rendering");
    if (!mat && !fused_supported(ctx->cfg.n1, ctx->cfg.n2))
        return fail(FPO_ERR_UNSUPPORTED, "the fused IDFT supports (n1, n2) in {(31,5), (11,5), (21,5), (31,11)}");

    DeviceGuard g(ctx->cfg.device);
    if (!g.ok) return fail(FPO_ERR_CUDA, "cudaSetDevice failed");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaError_t e;
    if (mat && ctx->table_leaves < ctx->n_leaves) {
        dfree(ctx->d_table);
        e = cudaMalloc((void **)&ctx->d_table, table_alloc_bytes(ctx));
        if (e != cudaSuccess) { ctx->table_leaves = 0; return cuda_fail(e, "cudaMalloc(table)"); }
        ctx->table_leaves = ctx->n_leaves;
    }
    auto rec = [&](int i) -> cudaError_t {
        return opts->events[i] ? cudaEventRecord((cudaEvent_t)opts->events[i], s) : cudaSuccess;
    };
    if ((e = rec(0)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    if (n_rays == 0) {
        if ((e = rec(1)) != cudaSuccess || (e = rec(2)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
        return FPO_OK;
    }
    if (mat && !((fl & FPO_FLAG_REUSE_TABLE) && ctx->table_ok && ctx->table_t == rays->t)) {
        ctx->table_ok = false;
        const int ce = launch_table_pass(ctx, rays->t, ctx->d_table, 0, s, 0, 0,
                                         (fl & FPO_FLAG_TEST_DEVICE_TIMEOUT) != 0);
        if (ce != cudaSuccess) return cuda_fail((cudaError_t)ce, "IDFT table launch");
        ctx->table_ok = (fl & FPO_FLAG_TEST_DEVICE_TIMEOUT) == 0;
        ctx->table_t = rays->t;
    }
    if ((e = rec(1)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");

    TraverseParams p = traverse_params(ctx, rays, opts, out_rgb, n_rays);
    const bool dbg = (fl & (FPO_FLAG_RECORD_VISITS | FPO_FLAG_OUT_T | FPO_FLAG_MARK_LEAVES |
                            FPO_FLAG_STATS)) != 0;
    int ce = launch_traverse(p, mat, dbg, ctx->sm_count, s);
    if (ce != cudaSuccess) return cuda_fail((cudaError_t)ce, "traverse launch");
    if ((e = rec(2)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    return FPO_OK;
}

int fpo_render_frames(fpo_ctx *ctx, const fpo_rays *frames, uint32_t n_frames, const fpo_frame_opts *opts,
                      float *out_rgb, void *const *frame_done, void *cuda_stream)
{
    if (!ctx || !opts || (n_frames && !frames)) return fail(FPO_ERR_INVALID_ARG, "NULL argument");
    if (!ctx->has_tree) return fail(FPO_ERR_NO_TREE, "render before fpo_upload_tree");
    if (opts->flags) return fail(FPO_ERR_INVALID_ARG, "fpo_render_frames takes no debug outputs (flags must be 0)");
    uint64_t R = 0;
    for (uint32_t k = 0; k < n_frames; ++k) {
        uint64_t nr = 0;
        const int st = check_rays(&frames[k], &nr);
        if (st != FPO_OK) return st;
        if (frames[k].mode == FPO_RAYS_EXPLICIT && frames[k].t_per_ray)
            return fail(FPO_ERR_INVALID_ARG, "per-ray times need fpo_render (fused IDFT)");
        if (k == 0) R = nr;
        else if (nr != R) return fail(FPO_ERR_INVALID_ARG, "every frame must have the same number of rays");
    }
    if (n_frames == 0 || R == 0) return FPO_OK;
    if (!out_rgb) return fail(FPO_ERR_INVALID_ARG, "out_rgb is NULL");
    if (!(opts->stop_T >= 0.0f)) return fail(FPO_ERR_INVALID_ARG, "stop_T must be >= 0");
    fpo_frame_opts o1 = *opts;
    for (int i = 0; i < 3; ++i) o1.events[i] = nullptr;
    const bool mat = ctx->cfg.idft_mode != FPO_IDFT_FUSED && ctx->n_leaves > 0;
    if (!mat || n_frames == 1) {
        for (uint32_t k = 0; k < n_frames; ++k) {
            const int st = fpo_render(ctx, &frames[k], &o1, out_rgb + (size_t)k * R * 3, cuda_stream);
            if (st != FPO_OK) return st;
            if (frame_done && frame_done[k]) {
                const cudaError_t e = cudaEventRecord((cudaEvent_t)frame_done[k], (cudaStream_t)cuda_stream);
                if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord(frame_done)");
            }
        }
        return FPO_OK;
    }
    if (ctx->cfg.storage == FPO_STORAGE_LATENT && !ctx->has_latents)
        return fail(FPO_ERR_INVALID_ARG, "LATENT storage: call fpo_set_latents before rendering");
    DeviceGuard g(ctx->cfg.device);
    if (!g.ok) return fail(FPO_ERR_CUDA, "cudaSetDevice failed");
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < FPO_PIPE_DEPTH; ++b) {
        float *&tb = b ? ctx->d_ptable[b] : ctx->d_table;
        size_t &tl = b ? ctx->ptable_leaves[b] : ctx->table_leaves;
        if (tl < ctx->n_leaves) {
            dfree(tb);
            e = cudaMalloc((void **)&tb, table_alloc_bytes(ctx));
            if (e != cudaSuccess) { tl = 0; return cuda_fail(e, "cudaMalloc(table)"); }
            tl = ctx->n_leaves;
        }
    }
    if (!ctx->aux || !ctx->trav[FPO_PIPE_DEPTH - 1] || !ctx->ev_trav[FPO_PIPE_DEPTH - 1]) {
        // created once; a failed attempt is retried whole
        if (!ctx->aux) e = cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking);
        if (e == cudaSuccess && !ctx->ev_entry) e = cudaEventCreateWithFlags(&ctx->ev_entry, cudaEventDisableTiming);
        for (int b = 0; b < FPO_PIPE_DEPTH && e == cudaSuccess; ++b) {
            if (b && !ctx->trav[b]) e = cudaStreamCreateWithFlags(&ctx->trav[b], cudaStreamNonBlocking);
            if (e == cudaSuccess && !ctx->ev_mat[b]) e = cudaEventCreateWithFlags(&ctx->ev_mat[b], cudaEventDisableTiming);
            if (e == cudaSuccess && !ctx->ev_trav[b]) e = cudaEventCreateWithFlags(&ctx->ev_trav[b], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return cuda_fail(e, "stream/event creation");
    }
    // Shapes that let both kernels be resident on an SM at once: the IDFT
    // pass in materialise_pipeline_shape, or for LATENT storage one 256-thread
    // decoder CTA (two warpgroup pipelines, 128 TMEM columns) per SM.
    bool overlap = true;
    MatShape mshape{};
    int carveout = 0;
    if (overlap) {
        int max_smem = 0, reserved = 0;
        if ((e = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, ctx->cfg.device)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, ctx->cfg.device)) != cudaSuccess)
            return cuda_fail(e, "cudaDeviceGetAttribute");
        if (ctx->cfg.storage == FPO_STORAGE_LATENT) {
            mshape.ctas_per_sm = 1;
            mshape.stages = 1;  // (a positive value selects the pipeline shape)
            mshape.smem_per_cta = latent_pipeline_smem_bytes();
        } else {
            mshape = materialise_pipeline_shape(ctx->cfg.storage, ctx->cfg.n1, ctx->cfg.n2, PIPE_MAT_SMEM_BUDGET);
            if (FPO_PIPE_MAT_CTAS > 0) mshape.ctas_per_sm = FPO_PIPE_MAT_CTAS;
        }
        const long need = (long)PIPE_TRAV_CTAS * (traverse_smem_bytes(ctx->n_smem_nodes, false, PIPE_TRAV_THREADS) + PIPE_STATIC_SMEM + reserved) +
                          (long)mshape.ctas_per_sm * (mshape.smem_per_cta + PIPE_STATIC_SMEM + reserved);
        // The driver rounds a carveout request up to one of the SM's shared-
        // memory configurations: ask for the smallest one that holds `need`.
        long config = -1;
        for (const int kb : SMEM_CONFIGS_KB)
            if ((long)kb * 1024 >= need) { config = (long)kb * 1024; break; }
        if (config < 0 || config > max_smem) overlap = false;
        else carveout = (int)(config * 100 / max_smem);
    }
    ctx->table_ok = false;  // the pipeline writes every slot's table
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // Frame k takes slot b = k mod depth: the slot's table and traversal
    // stream (slot 0: d_table and the caller's stream) and tile counter.  The
    // table passes run in order on the auxiliary stream, ahead of the
    // traversals; the traversals of consecutive frames run on different
    // streams, so that the next ones fill the SMs that the last warps of the
    // earlier ones leave idle.  Table b is rewritten only after the
    // traversal that read it (event ev_trav[b]), and the caller's stream
    // waits for every slot's last traversal at the end.
    if ((e = cudaEventRecord(ctx->ev_entry, s)) != cudaSuccess || (e = cudaStreamWaitEvent(ctx->aux, ctx->ev_entry, 0)) != cudaSuccess)
        return cuda_fail(e, "stream ordering");
    for (int b = 1; b < FPO_PIPE_DEPTH; ++b)
        if ((e = cudaStreamWaitEvent(ctx->trav[b], ctx->ev_entry, 0)) != cudaSuccess) return cuda_fail(e, "stream ordering");
    // Views of one frame time (every t bit-equal): one table pass, and every
    // traversal of the call reads that table (nothing rewrites it before the
    // call's end, after which the caller's stream has waited for them all).
    bool one_t = n_frames > 1;
    for (uint32_t k = 1; k < n_frames && one_t; ++k)
        one_t = memcmp(&frames[k].t, &frames[0].t, sizeof(double)) == 0;
    for (uint32_t k = 0; k < n_frames; ++k) {
        const int b = (int)(k % FPO_PIPE_DEPTH);
        float *tbl = one_t ? ctx->d_table : (b ? ctx->d_ptable[b] : ctx->d_table);
        cudaStream_t ts = FPO_PIPE_SLOT_STREAMS && b ? ctx->trav[b] : s;
        int ce = cudaSuccess;
        if (!one_t || k == 0) {
            if (k >= FPO_PIPE_DEPTH && (e = cudaStreamWaitEvent(ctx->aux, ctx->ev_trav[b], 0)) != cudaSuccess)
                return cuda_fail(e, "wait");
            ce = overlap ? launch_table_pass(ctx, frames[k].t, tbl, mshape.ctas_per_sm, ctx->aux, mshape.stages, carveout, false)
                         : launch_table_pass(ctx, frames[k].t, tbl, 0, ctx->aux, 0, 0, false);
            if (ce != cudaSuccess) return cuda_fail((cudaError_t)ce, "IDFT table launch");
            if ((e = cudaEventRecord(ctx->ev_mat[b], ctx->aux)) != cudaSuccess)
                return cuda_fail(e, "stream ordering");
        }
        if ((e = cudaStreamWaitEvent(ts, ctx->ev_mat[one_t ? 0 : b], 0)) != cudaSuccess)
            return cuda_fail(e, "stream ordering");
        TraverseParams p = traverse_params(ctx, &frames[k], &o1, out_rgb + (size_t)k * R * 3, R);
        p.table = reinterpret_cast<const float4 *>(tbl);
        p.tiles = ctx->d_status + 1 + (FPO_PIPE_SLOT_STREAMS ? 2 * b : 0);  // this slot's tile counter and finished warps
        if (overlap) {
            p.block_threads = PIPE_TRAV_THREADS;
            p.max_ctas_per_sm = PIPE_TRAV_CTAS;
            p.carveout = carveout;
        }
        ce = launch_traverse(p, true, false, ctx->sm_count, ts);
        if (ce != cudaSuccess) return cuda_fail((cudaError_t)ce, "traverse launch");
        if ((e = cudaEventRecord(ctx->ev_trav[b], ts)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
        if (frame_done && frame_done[k] && (e = cudaEventRecord((cudaEvent_t)frame_done[k], ts)) != cudaSuccess)
            return cuda_fail(e, "cudaEventRecord(frame_done)");
    }
    // everything above is ordered before the caller's later work
    for (uint32_t b = 1; b < FPO_PIPE_DEPTH && b < n_frames; ++b)
        if ((e = cudaStreamWaitEvent(s, ctx->ev_trav[b], 0)) != cudaSuccess) return cuda_fail(e, "stream ordering");
    return FPO_OK;
}

int fpo_render_backward(fpo_ctx *ctx, const fpo_rays *rays, const fpo_frame_opts *opts,
                        const float *out_rgb, const float *dL_drgb, float *dL_dcoeffs,
                        void *cuda_stream)
{
    if (!ctx || !rays || !opts) return fail(FPO_ERR_INVALID_ARG, "NULL argument");
    if (!ctx->has_tree) return fail(FPO_ERR_NO_TREE, "backward before fpo_upload_tree");
    uint64_t n_rays = 0;
    int st = check_rays(rays, &n_rays);
    if (st != FPO_OK) return st;
    if (ctx->cfg.storage != FPO_STORAGE_F32)
        return fail(FPO_ERR_UNSUPPORTED, "gradients are taken with respect to FP32 records only");
    if (!fused_supported(ctx->cfg.n1, ctx->cfg.n2))
        return fail(FPO_ERR_UNSUPPORTED, "the adjoint supports (n1, n2) in {(31,5), (11,5), (21,5), (31,11)}");
    if (n_rays > 0 && (!out_rgb || !dL_drgb)) return fail(FPO_ERR_INVALID_ARG, "out_rgb and dL_drgb must be non-NULL");
    if (ctx->n_leaves > 0 && !dL_dcoeffs) return fail(FPO_ERR_INVALID_ARG, "dL_dcoeffs is NULL");
    const bool fp64 = (opts->flags & FPO_FLAG_FP64_GRADCHECK) != 0;
    if (reinterpret_cast<uintptr_t>(dL_dcoeffs) % (fp64 ? 8 : 16) != 0)
        return fail(FPO_ERR_INVALID_ARG, fp64 ? "dL_dcoeffs must be 8-byte aligned" : "dL_dcoeffs must be 16-byte aligned");
    if (!(opts->stop_T >= 0.0f)) return fail(FPO_ERR_INVALID_ARG, "stop_T must be >= 0");
    if (n_rays == 0 || ctx->n_leaves == 0) return FPO_OK;
    DeviceGuard g(ctx->cfg.device);
    if (!g.ok) return fail(FPO_ERR_CUDA, "cudaSetDevice failed");
    const bool mark = (opts->flags & FPO_FLAG_MARK_LEAVES) != 0;
    if (mark && !opts->leaf_mark) return fail(FPO_ERR_INVALID_ARG, "FPO_FLAG_MARK_LEAVES needs leaf_mark");
    fpo_frame_opts o = *opts;
    o.flags = 0;  // the other debug outputs belong to the forward
    BackwardParams q{};
    q.tp = traverse_params(ctx, rays, &o, nullptr, n_rays);
    q.out_rgb = out_rgb;
    q.dL_drgb = dL_drgb;
    q.dL_dcoeffs = fp64 ? nullptr : dL_dcoeffs;
    q.dL_dcoeffs64 = fp64 ? reinterpret_cast<double *>(dL_dcoeffs) : nullptr;
    q.leaf_mark = mark ? opts->leaf_mark : nullptr;
    const int ce = launch_backward(q, ctx->sm_count, cuda_stream);
    if (ce != cudaSuccess) return cuda_fail((cudaError_t)ce, "backward launch");
    return FPO_OK;
}

int fpo_set_latents(fpo_ctx *ctx, const uint16_t *latents, const fpo_decoder *dec, void *cuda_stream)
{
    if (!ctx || !dec) return fail(FPO_ERR_INVALID_ARG, "NULL argument");
    if (!ctx->has_tree) return fail(FPO_ERR_NO_TREE, "set_latents before fpo_upload_tree");
    if (ctx->cfg.storage != FPO_STORAGE_LATENT) return fail(FPO_ERR_UNSUPPORTED, "context storage is not LATENT");
    if (!dec->w1 || !dec->b1 || !dec->w2 || !dec->b2 || !dec->w3 || !dec->b3 || (ctx->n_leaves && !latents))
        return fail(FPO_ERR_INVALID_ARG, "NULL array");
    ctx->table_ok = false;  // the coefficients change
    DeviceGuard g(ctx->cfg.device);
    if (!g.ok) return fail(FPO_ERR_CUDA, "cudaSetDevice failed");
    const int nc = ctx->cfg.n1 + 27 * ctx->cfg.n2;
    const size_t nw = 64 * 32 + 64 * 64 + (size_t)nc * 64, nb = 64 + 64 + (size_t)nc;
    cudaError_t e = cudaSuccess;
    if (!ctx->d_dec_w) e = cudaMalloc((void **)&ctx->d_dec_w, nw * 2);
    if (e == cudaSuccess && !ctx->d_dec_b) e = cudaMalloc((void **)&ctx->d_dec_b, nb * 4);
    if (e == cudaSuccess && !ctx->d_latents && ctx->n_leaves)
        e = cudaMalloc((void **)&ctx->d_latents, (size_t)ctx->n_leaves * 64);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(latents)");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    struct { void *dst; const void *src; size_t bytes; } cp[6] = {
        {ctx->d_dec_w, dec->w1, 64 * 32 * 2}, {ctx->d_dec_w + 64 * 32, dec->w2, 64 * 64 * 2},
        {ctx->d_dec_w + 64 * 32 + 64 * 64, dec->w3, (size_t)nc * 64 * 2}, {ctx->d_dec_b, dec->b1, 64 * 4},
        {ctx->d_dec_b + 64, dec->b2, 64 * 4}, {ctx->d_dec_b + 128, dec->b3, (size_t)nc * 4}};
    for (auto &c : cp) {
        e = cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "decoder copy");
    }
    const int ce = launch_gather_rows(latents, ctx->d_latents, ctx->d_perm, ctx->n_leaves, 64, ctx->sm_count, s);
    if (ce != cudaSuccess) return cuda_fail((cudaError_t)ce, "latent gather");
    ctx->has_latents = true;
    return FPO_OK;
}

int fpo_set_coeffs(fpo_ctx *ctx, const float *coeffs, void *cuda_stream)
{
    if (!ctx) return fail(FPO_ERR_INVALID_ARG, "ctx is NULL");
    if (!ctx->has_tree) return fail(FPO_ERR_NO_TREE, "set_coeffs before fpo_upload_tree");
    if (ctx->cfg.storage != FPO_STORAGE_F32)
        return fail(FPO_ERR_UNSUPPORTED, "in-place coefficient updates need FP32 storage");
    if (ctx->n_leaves == 0) return FPO_OK;
    if (!coeffs) return fail(FPO_ERR_INVALID_ARG, "coeffs is NULL");
    ctx->table_ok = false;  // the coefficients change
    DeviceGuard g(ctx->cfg.device);
    if (!g.ok) return fail(FPO_ERR_CUDA, "cudaSetDevice failed");
    const int ce = launch_set_coeffs(coeffs, ctx->d_perm, static_cast<float *>(ctx->d_sig),
                                     static_cast<float *>(ctx->d_z), ctx->n_leaves, ctx->cfg.n1,
                                     ctx->cfg.n2, ctx->sm_count, cuda_stream);
    if (ce != cudaSuccess) return cuda_fail((cudaError_t)ce, "set_coeffs launch");
    return FPO_OK;
}

int fpo_set_coeffs_from_decoder(fpo_ctx *ctx, const fpo_mlp *w, const float *latents, uint32_t flags, void *cuda_stream)
{
    if (!ctx) return fail(FPO_ERR_INVALID_ARG, "ctx is NULL");
    if (!ctx->has_tree) return fail(FPO_ERR_NO_TREE, "set_coeffs_from_decoder before fpo_upload_tree");
    if (ctx->cfg.storage != FPO_STORAGE_F32)
        return fail(FPO_ERR_UNSUPPORTED, "in-place coefficient updates need FP32 storage");
    if (!w || !w->w1 || !w->b1 || !w->w2 || !w->b2 || !w->w3 || !w->b3) return fail(FPO_ERR_INVALID_ARG, "NULL weights");
    if (ctx->cfg.n1 + 27 * ctx->cfg.n2 > decoder_grad_max_coeffs())
        return fail(FPO_ERR_UNSUPPORTED, "n1 + 27 n2 above the decoder's 176 outputs");
    if (ctx->n_leaves == 0) return FPO_OK;
    if (!latents) return fail(FPO_ERR_INVALID_ARG, "latents is NULL");
    if (flags & ~(uint32_t)(FPO_FLAG_TENSOR_CORES | FPO_FLAG_TEST_DEVICE_TIMEOUT))
        return fail(FPO_ERR_INVALID_ARG, "unknown flags");
    ctx->table_ok = false;  // the coefficients change
    DeviceGuard g(ctx->cfg.device);
    if (!g.ok) return fail(FPO_ERR_CUDA, "cudaSetDevice failed");
    const int ce = (flags & FPO_FLAG_TENSOR_CORES)
                       ? launch_decode_records_tc(*w, ctx->cfg.n1, ctx->cfg.n2, ctx->n_leaves, latents, ctx->d_perm,
                                                  static_cast<float *>(ctx->d_sig), static_cast<float *>(ctx->d_z),
                                                  ctx->d_status, (flags & FPO_FLAG_TEST_DEVICE_TIMEOUT) != 0,
                                                  ctx->sm_count, cuda_stream)
                       : launch_decode_records(*w, ctx->cfg.n1, ctx->cfg.n2, ctx->n_leaves, latents, ctx->d_perm,
                                               static_cast<float *>(ctx->d_sig), static_cast<float *>(ctx->d_z),
                                               ctx->sm_count, cuda_stream);
    if (ce != cudaSuccess) return cuda_fail((cudaError_t)ce, "decode launch");
    return FPO_OK;
}

int fpo_adam_leaves(fpo_ctx *ctx, float *param, float *grad, float *m, float *v, uint8_t *leaf_mark, float lr,
                    float beta1, float beta2, float eps, uint32_t step, void *cuda_stream)
{
    if (!ctx) return fail(FPO_ERR_INVALID_ARG, "ctx is NULL");
    if (!ctx->has_tree) return fail(FPO_ERR_NO_TREE, "adam_leaves before fpo_upload_tree");
    if (ctx->cfg.storage != FPO_STORAGE_F32)
        return fail(FPO_ERR_UNSUPPORTED, "in-place coefficient updates need FP32 storage");
    if (ctx->n_leaves == 0) return FPO_OK;
    if (!param || !grad || !m || !v || !leaf_mark) return fail(FPO_ERR_INVALID_ARG, "NULL array");
    if (step < 1) return fail(FPO_ERR_INVALID_ARG, "step counts from 1");
    if (!(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
        return fail(FPO_ERR_INVALID_ARG, "lr >= 0, beta in [0, 1), eps > 0");
    ctx->table_ok = false;  // the coefficients change
    DeviceGuard g(ctx->cfg.device);
    if (!g.ok) return fail(FPO_ERR_CUDA, "cudaSetDevice failed");
    LeafAdamParams p{};
    p.param = param;
    p.grad = grad;
    p.m = m;
    p.v = v;
    p.leaf_mark = leaf_mark;
    p.perm = ctx->d_perm;
    p.sig = static_cast<float *>(ctx->d_sig);
    p.zc = static_cast<float *>(ctx->d_z);
    p.n_leaves = ctx->n_leaves;
    p.n1 = ctx->cfg.n1;
    p.n2 = ctx->cfg.n2;
    p.sig_stride = sig_stride(ctx->cfg.n1);
    p.z_stride = z_stride(ctx->cfg.n2);
    p.lr = lr;
    p.beta1 = beta1;
    p.beta2 = beta2;
    p.eps = eps;
    p.bc1 = (float)(1.0 - std::pow((double)beta1, (double)step));
    p.bc2 = (float)(1.0 - std::pow((double)beta2, (double)step));
    const int ce = launch_leaf_adam(p, ctx->sm_count, cuda_stream);
    if (ce != cudaSuccess) return cuda_fail((cudaError_t)ce, "adam_leaves launch");
    return FPO_OK;
}

int fpo_dft_leaves(int32_t n1, int32_t n2, uint32_t n_frames, uint32_t n_leaves, const float *values,
                   float *coeffs, uint32_t *status, uint32_t flags, void *cuda_stream)
{
    if (n1 < 1 || n1 > 32 || n2 < 1 || n2 > 16) return fail(FPO_ERR_INVALID_ARG, "n1 in [1, 32], n2 in [1, 16]");
    if (flags & ~(uint32_t)FPO_FLAG_TEST_DEVICE_TIMEOUT) return fail(FPO_ERR_INVALID_ARG, "unknown flags");
    if (n_frames < 1 || n_frames > 256) return fail(FPO_ERR_INVALID_ARG, "n_frames must be in [1, 256]");
    if (n_leaves == 0) return FPO_OK;
    if (!values || !coeffs) return fail(FPO_ERR_INVALID_ARG, "NULL array");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device query");
    const int ce = launch_dft(values, coeffs, n_leaves, n1, n2, (int)n_frames, status,
                              (flags & FPO_FLAG_TEST_DEVICE_TIMEOUT) != 0, sms, cuda_stream);
    if (ce != cudaSuccess) return cuda_fail((cudaError_t)ce, "dft launch");
    return FPO_OK;
}

int fpo_status_sync(fpo_ctx *ctx, void *cuda_stream)
{
    if (!ctx) return fail(FPO_ERR_INVALID_ARG, "ctx is NULL");
    DeviceGuard g(ctx->cfg.device);
    if (!g.ok) return fail(FPO_ERR_CUDA, "cudaSetDevice failed");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    uint32_t st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, ctx->d_status, sizeof st, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    if (st) {
        e = cudaMemsetAsync(ctx->d_status, 0, sizeof st, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "status clear");
    }
    if (st & STATUS_TRAVERSAL_LIMIT) return fail(FPO_ERR_TRAVERSAL_LIMIT, "a ray exceeded its step cap");
    if (st & STATUS_VISIT_OVERFLOW) return fail(FPO_ERR_VISIT_OVERFLOW, "a ray had more visits than visit_cap");
    if (st & STATUS_DEVICE_TIMEOUT) return fail(FPO_ERR_DEVICE_TIMEOUT, "a device-side wait gave up after its time limit");
    if (st & STATUS_FP16_RANGE)
        return fail(FPO_ERR_RANGE, "a latent decoder weight, bias or hidden activation exceeded the FP16 range (65504)");
    return FPO_OK;
}

void fpo_destroy(fpo_ctx *ctx)
{
    if (!ctx) return;
    {
        DeviceGuard g(ctx->cfg.device);
        ctx->free_tree();
        dfree(ctx->d_status);
        if (ctx->aux) cudaStreamDestroy(ctx->aux);
        if (ctx->ev_entry) cudaEventDestroy(ctx->ev_entry);
        for (int b = 0; b < PIPE_MAX; ++b) {
            if (ctx->trav[b]) cudaStreamDestroy(ctx->trav[b]);
            if (ctx->ev_mat[b]) cudaEventDestroy(ctx->ev_mat[b]);
            if (ctx->ev_trav[b]) cudaEventDestroy(ctx->ev_trav[b]);
        }
    }
    delete ctx;
}

}  // extern "C"
