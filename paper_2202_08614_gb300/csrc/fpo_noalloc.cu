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
    // the same rays and options as fpo_render accepts, minus per-ray times
    if (rays->mode == FPO_RAYS_EXPLICIT && rays->t_per_ray)
        return set_last_error(FPO_ERR_INVALID_ARG, "per-ray times need fpo_render (fused IDFT)");
    uint64_t n_rays = 0;
    int st = check_rays(rays, &n_rays);
    if (st != FPO_OK) return st;
    if ((st = check_render_opts(ctx, opts, n_rays, out_rgb)) != FPO_OK) return st;
    const uint32_t fl = opts->flags;

    CurrentDevice g(c.device);
    if (!g.ok) return set_last_error(FPO_ERR_CUDA, "cudaSetDevice failed");
    float *table = nullptr;
    st = table_address(c.device, &table);
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
        const int ce = launch_table_pass(ctx, rays->t, table, 0, s, 0, 0, (fl & FPO_FLAG_TEST_DEVICE_TIMEOUT) != 0);
        if (ce != cudaSuccess) return cuda_err((cudaError_t)ce, "IDFT table launch");
    }
    if ((e = rec(1)) != cudaSuccess) return cuda_err(e, "cudaEventRecord");
    TraverseParams p = traverse_params(ctx, rays, opts, out_rgb, n_rays);
    p.table = reinterpret_cast<const float4 *>(table);
    const bool dbg = (fl & (FPO_FLAG_RECORD_VISITS | FPO_FLAG_OUT_T | FPO_FLAG_MARK_LEAVES | FPO_FLAG_STATS)) != 0;
    const int ce = launch_traverse(p, mat, dbg, c.sm_count, s);
    if (ce != cudaSuccess) return cuda_err((cudaError_t)ce, "traverse launch");
    if ((e = rec(2)) != cudaSuccess) return cuda_err(e, "cudaEventRecord");
    return FPO_OK;
}
