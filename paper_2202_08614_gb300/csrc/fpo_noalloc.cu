// fpo_render_noalloc: the materialised-mode render of fpo_render for callers
// that cannot allocate device memory.  The per-frame IDFT table (the only
// scratch of that path beyond the context's status words) lives in a
// file-scope __device__ array instead of a cudaMalloc'd buffer.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "fpo_internal.h"

using namespace fpo;

namespace {
constexpr uint32_t NOALLOC_MAX_LEAVES = 65536;  // 65536 x 128 B = 8 MiB per GPU
}

// Shared by every call on a device; holds the last call's table until the
// process exits.  Calls whose kernels overlap on the GPU race on it.
static __device__ __align__(256) float g_noalloc_table[(size_t)NOALLOC_MAX_LEAVES * TABLE_STRIDE];

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
float *g_table_addr[MAX_DEVICES] = {};

// Device address of g_noalloc_table on `dev` (which must be current).  The
// host-side name of the array is only a stand-in, so the address is looked
// up once per device and cached.
int table_address(int dev, float **out)
{
    if (dev < 0 || dev >= MAX_DEVICES) return set_last_error(FPO_ERR_INVALID_ARG, "device ordinal too large");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_table_addr[dev]) {
        float *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress((void **)&ptr, g_noalloc_table);
        if (e != cudaSuccess || !ptr) {
            char buf[256];
            std::snprintf(buf, sizeof buf, "cudaGetSymbolAddress(table): %s", cudaGetErrorString(e));
            return set_last_error(FPO_ERR_CUDA, buf);
        }
        g_table_addr[dev] = ptr;
    }
    *out = g_table_addr[dev];
    return FPO_OK;
}

struct CurrentDevice {
    int prev = -1;
    bool ok = false;
    explicit CurrentDevice(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~CurrentDevice()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" int fpo_render_noalloc(fpo_ctx *ctx, const fpo_rays *rays, const fpo_frame_opts *opts,
                                  float *out_rgb, void *cuda_stream)
{
    if (!ctx || !rays || !opts) return set_last_error(FPO_ERR_INVALID_ARG, "NULL argument");
    const CtxView c = ctx_view(ctx);
    if (!c.has_tree) return set_last_error(FPO_ERR_NO_TREE, "render before fpo_upload_tree");
    if (c.storage == FPO_STORAGE_LATENT)
        return set_last_error(FPO_ERR_UNSUPPORTED, "fpo_render_noalloc renders stored coefficients, not LATENT storage");
    if (c.n_leaves > NOALLOC_MAX_LEAVES) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "tree has %u leaves; fpo_render_noalloc supports at most %u",
                      c.n_leaves, NOALLOC_MAX_LEAVES);
        return set_last_error(FPO_ERR_INVALID_ARG, buf);
    }
    uint64_t n_rays = 0;
    if (rays->mode == FPO_RAYS_CAMERA) {
        if (!(rays->fov_y_deg > 0.0 && rays->fov_y_deg < 180.0))
            return set_last_error(FPO_ERR_INVALID_ARG, "fov_y_deg must be in (0, 180)");
        double f[3], x[3];
        for (int k = 0; k < 3; ++k) f[k] = rays->target[k] - rays->eye[k];
        x[0] = f[1] * rays->up[2] - f[2] * rays->up[1];
        x[1] = f[2] * rays->up[0] - f[0] * rays->up[2];
        x[2] = f[0] * rays->up[1] - f[1] * rays->up[0];
        if (!(f[0] * f[0] + f[1] * f[1] + f[2] * f[2] > 0.0) || !(x[0] * x[0] + x[1] * x[1] + x[2] * x[2] > 0.0))
            return set_last_error(FPO_ERR_INVALID_ARG, "degenerate camera");
        n_rays = (uint64_t)rays->width * rays->height;
    } else if (rays->mode == FPO_RAYS_EXPLICIT) {
        if (rays->t_per_ray) return set_last_error(FPO_ERR_INVALID_ARG, "per-ray times need fpo_render (fused IDFT)");
        if (rays->n > 0 && (!rays->o || !rays->d)) return set_last_error(FPO_ERR_INVALID_ARG, "o and d must be non-NULL");
        n_rays = rays->n;
    } else {
        return set_last_error(FPO_ERR_INVALID_ARG, "unknown ray mode");
    }
    if (n_rays >= (1ull << 31)) return set_last_error(FPO_ERR_INVALID_ARG, "too many rays");
    if (n_rays > 0 && !out_rgb) return set_last_error(FPO_ERR_INVALID_ARG, "out_rgb is NULL");
    const uint32_t fl = opts->flags;
    if ((fl & FPO_FLAG_RECORD_VISITS) && (!opts->visit_count || (opts->visit_cap && !opts->visit_log)))
        return set_last_error(FPO_ERR_INVALID_ARG, "RECORD_VISITS needs visit_count (and visit_log)");
    if ((fl & FPO_FLAG_OUT_T) && !opts->out_T) return set_last_error(FPO_ERR_INVALID_ARG, "OUT_T needs out_T");
    if ((fl & FPO_FLAG_MARK_LEAVES) && !opts->leaf_mark && c.n_leaves)
        return set_last_error(FPO_ERR_INVALID_ARG, "MARK_LEAVES needs leaf_mark");
    if ((fl & FPO_FLAG_STATS) && !opts->stats) return set_last_error(FPO_ERR_INVALID_ARG, "STATS needs stats");
    if (!(opts->stop_T >= 0.0f)) return set_last_error(FPO_ERR_INVALID_ARG, "stop_T must be >= 0");

    CurrentDevice g(c.device);
    if (!g.ok) return set_last_error(FPO_ERR_CUDA, "cudaSetDevice failed");
    float *table = nullptr;
    int st = table_address(c.device, &table);
    if (st != FPO_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    auto rec = [&](int i) -> cudaError_t {
        return opts->events[i] ? cudaEventRecord((cudaEvent_t)opts->events[i], s) : cudaSuccess;
    };
    auto cuda_err = [&](cudaError_t e, const char *what) {
        char buf[256];
        std::snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
        return set_last_error(FPO_ERR_CUDA, buf);
    };
    cudaError_t e;
    if ((e = rec(0)) != cudaSuccess) return cuda_err(e, "cudaEventRecord");
    if (n_rays == 0) {
        if ((e = rec(1)) != cudaSuccess || (e = rec(2)) != cudaSuccess) return cuda_err(e, "cudaEventRecord");
        return FPO_OK;
    }
    const bool mat = c.n_leaves > 0;
    if (mat) {
        // Every table entry the traversal reads is written first: nothing to clear.
        MaterialiseParams mp{};
        const RecordLayout L = record_layout(c.storage, c.n1, c.n2);
        mp.sig = c.d_sig;
        mp.zc = c.d_z;
        mp.scale = c.d_scale;
        mp.table = table;
        mp.n_leaves = c.n_leaves;
        mp.storage = c.storage;
        mp.n1 = c.n1;
        mp.n2 = c.n2;
        mp.sig_stride = L.sig_elems;
        mp.z_stride = L.z_elems;
        mp.stages = materialise_stages(c.storage, c.n1, c.n2);
        mp.max_ctas_per_sm = 0;
        mp.half_table = c.half_table;
        mp.t = rays->t;
        mp.period_T = c.period_T;
        mp.status = c.d_status;
        const int ce = launch_materialise(mp, c.sm_count, s);
        if (ce != cudaSuccess) return cuda_err((cudaError_t)ce, "materialise launch");
    }
    if ((e = rec(1)) != cudaSuccess) return cuda_err(e, "cudaEventRecord");
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
    p.fr.period_T = c.period_T;
    p.fr.ro = rays->o;
    p.fr.rd = rays->d;
    p.fr.rt = nullptr;
    p.nodes = c.d_nodes;
    p.root_kind = c.root_kind;
    p.depth = c.depth;
    p.n_smem_nodes = c.n_smem_nodes;
    p.grid_scale = (float)((double)(1u << c.depth) / c.aabb_size);
    for (int k = 0; k < 3; ++k) p.amin[k] = (float)c.aabb_min[k];
    p.table = reinterpret_cast<const float4 *>(table);
    p.half_table = c.half_table;
    p.sig = reinterpret_cast<const float4 *>(c.d_sig);
    p.zc = static_cast<const float *>(c.d_z);
    p.n1 = c.n1;
    p.n2 = c.n2;
    p.sig_stride4 = sig_stride(c.n1) / 4;
    p.z_stride = z_stride(c.n2);
    for (int k = 0; k < 3; ++k) p.bg[k] = opts->bg[k];
    p.stop_T = opts->stop_T;
    p.flags = fl;
    p.out_rgb = out_rgb;
    p.out_T = opts->out_T;
    p.visit_log = opts->visit_log;
    p.visit_cap = opts->visit_cap;
    p.visit_count = opts->visit_count;
    p.leaf_mark = opts->leaf_mark;
    p.perm = c.d_perm;
    p.status = c.d_status;
    if (rays->mode == FPO_RAYS_CAMERA) {
        p.tiles_x = (rays->width + TILE_W - 1) / TILE_W;
        p.n_tiles = p.tiles_x * ((rays->height + TILE_H - 1) / TILE_H);
    } else {
        p.tiles_x = 0;
        p.n_tiles = (uint32_t)((n_rays + 31) / 32);
    }
    p.max_steps = c.max_steps > 0 ? (uint32_t)c.max_steps : 3u * (1u << c.depth) + 16u;
    p.block_threads = c.traverse_threads ? c.traverse_threads : 256;
    p.refill_min = c.refill_min ? (uint32_t)c.refill_min : 32u;
    p.inner_steps = c.inner_steps ? (uint32_t)c.inner_steps : 0xffffffffu;
    p.stats = reinterpret_cast<unsigned long long *>(opts->stats);
    const bool dbg = (fl & (FPO_FLAG_RECORD_VISITS | FPO_FLAG_OUT_T | FPO_FLAG_MARK_LEAVES | FPO_FLAG_STATS)) != 0;
    const int ce = launch_traverse(p, mat, dbg, c.sm_count, s);
    if (ce != cudaSuccess) return cuda_err((cudaError_t)ce, "traverse launch");
    if ((e = rec(2)) != cudaSuccess) return cuda_err(e, "cudaEventRecord");
    return FPO_OK;
}
