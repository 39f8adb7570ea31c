// Internal declarations shared by the host packer, the ABI layer and the
// CUDA kernels of the FPO renderer.  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda.h>  // CUtensorMap (a header type; nothing links the driver library)
#include <vector_types.h>

#include "fpo.h"

namespace fpo {

// ---------------------------------------------------------------------------
// Node array (breadth-first).  One node = 8 child slots of 32 bits = 32 bytes,
// one L2 sector.  Slot values: 0 = empty space, LEAF_BIT | i = leaf with
// internal index i, otherwise the index (>= 1) of an internal child node.
// The root is node 0 and is never referenced from a slot; its own kind is
// passed separately (ROOT_*).  Child c of a node covers the octant with
// bit 0 = x, bit 1 = y, bit 2 = z of the next level's coordinates.
constexpr uint32_t LEAF_BIT = 0x80000000u;
constexpr uint32_t ROOT_EMPTY = 0, ROOT_LEAF = 1, ROOT_NODE = 2;
constexpr int MAX_DEPTH = 12;

// Leaf records.  FP32 storage: a density record of SIG_STRIDE(n1) floats
// (n1 rounded up to a multiple of 4, 128 bytes for n1 = 31) and an SH record
// of Z_STRIDE(n2) floats (27 n2 rounded up to a multiple of 4), both arrays
// indexed by internal leaf index (breadth-first order, siblings adjacent).
inline int sig_stride(int n1) { return (n1 + 3) & ~3; }
inline int z_stride(int n2) { return (27 * n2 + 3) & ~3; }

// Stored record layout for any storage precision: element counts padded so
// that each record is a multiple of 16 bytes (bulk-copy granularity).  FP32
// gives sig_stride / z_stride above.  FP8 adds one FP32 scale per leaf in a
// separate array (codes are coefficient / scale).
struct RecordLayout {
    int sig_elems, z_elems, elem_bytes;
    bool scaled;
    int sig_bytes() const { return sig_elems * elem_bytes; }
    int z_bytes() const { return z_elems * elem_bytes; }
};
inline RecordLayout record_layout(int storage, int n1, int n2)
{
    const int eb = storage == FPO_STORAGE_F32 ? 4 : (storage == FPO_STORAGE_FP8_E4M3 ? 1 : 2);
    const int per16 = 16 / eb;
    RecordLayout L;
    L.elem_bytes = eb;
    L.sig_elems = (n1 + per16 - 1) / per16 * per16;
    L.z_elems = (27 * n2 + per16 - 1) / per16 * per16;
    L.scaled = storage == FPO_STORAGE_FP8_E4M3;
    return L;
}

// Host encoders (round to nearest even) from the format definitions:
// bfloat16 (1-8-7), IEEE binary16 (1-5-10, overflow to infinity) and
// FP8 E4M3 (1-4-3, bias 7, no infinities, saturating at +-448).
uint16_t encode_bf16(float x);
uint16_t encode_f16(float x);
uint8_t encode_e4m3(float x);

// Per-frame IDFT table: one 128-byte record per leaf,
// [sigma(t) clamped at 0, z_{c,k}(t) for c = 0..2, k = 0..8 (27 values), 4 zeros].
constexpr int TABLE_STRIDE = 32;

// Camera rays are scheduled in warp tiles of TILE_W x TILE_H pixels.
#ifndef FPO_TILE_W
#define FPO_TILE_W 4
#endif
constexpr int TILE_W = FPO_TILE_W, TILE_H = 32 / FPO_TILE_W;
static_assert(TILE_W * TILE_H == 32, "a tile is one warp of rays");

// Device status word bits.
constexpr uint32_t STATUS_TRAVERSAL_LIMIT = 1u, STATUS_VISIT_OVERFLOW = 2u, STATUS_DEVICE_TIMEOUT = 4u,
                   STATUS_FP16_RANGE = 8u;
// Limit of the waits that FPO_FLAG_TEST_DEVICE_TIMEOUT makes run out: 1 ms.
constexpr uint64_t TEST_WAIT_LIMIT_NS = 1000000ull;

struct PackedTree {
    uint32_t root_kind = ROOT_EMPTY;
    int depth = 0;                 // grid depth D: finest cell = 1 / 2^D of the cube
    std::vector<uint32_t> nodes;   // [n_nodes * 8]
    std::vector<uint32_t> perm;    // internal leaf index -> upload index
};

// Validates a tree description (and packs it when `out` is non-null).
// Returns FPO_OK, FPO_ERR_INVALID_ARG or FPO_ERR_BAD_TREE (message in *err).
int validate_and_pack(const fpo_tree_desc *tree, int n1, int n2, PackedTree *out,
                      std::string *err);

// ---------------------------------------------------------------------------
// Kernel parameters.

struct FrameParams {
    int mode;                 // FPO_RAYS_*
    uint32_t width, height, n_rays;
    double eye[3], target[3], up[3];
    double fov_y_deg;
    double t, period_T;
    const float *ro, *rd, *rt; // explicit rays (device)
};

struct TraverseParams {
    FrameParams fr;
    // tree
    const uint32_t *nodes;
    uint32_t root_kind;
    int depth;
    uint32_t n_smem_nodes;
    float grid_scale;         // 2^D / aabb_size
    float amin[3];
    double grid_scale64, amin64[3];  // the same in FP64 (gradient-check replay)
    // leaf data
    const float4 *table;      // per-frame IDFT table (materialised mode)
    int half_table;           // the table holds FP16 (64-byte lines) instead of FP32 (128-byte lines)
    const float4 *sig;        // density coefficient records (fused mode)
    const float *zc;          // SH coefficient records (fused mode)
    int n1, n2, sig_stride4, z_stride;
    // options and outputs
    float bg[3];
    float stop_T;
    uint32_t flags;
    float *out_rgb;
    float *out_T;
    uint32_t *visit_log;
    uint32_t visit_cap;
    uint32_t *visit_count;
    uint8_t *leaf_mark;
    const uint32_t *perm;
    // scheduling
    uint32_t *status;         // status bits (atomicOr)
    uint32_t *tiles;          // [0] tile counter, [1] finished warps (reset by the last warp)
    uint32_t n_tiles, tiles_x;
    uint32_t max_steps;
    uint32_t refill_min;      // warp refills its idle lanes once this many are idle (32: whole tiles)
    uint32_t inner_steps;     // steps a lane takes between two refill checks
    int block_threads;        // 128 or 256
    int max_ctas_per_sm;      // 0: as many as fit
    int carveout;             // preferred shared-memory carveout in percent (0: the driver's default)
    unsigned long long *stats; // FPO_FLAG_STATS: [steps, leaf visits, rays entering the tree]
};

struct MaterialiseParams {
    const void *sig;          // [n_leaves] records of sig_stride elements
    const void *zc;           // [n_leaves] records of z_stride elements
    const float *scale;       // [n_leaves] (FP8 storage) or nullptr
    float *table;             // [n_leaves][32] FP32, or [n_leaves][32] FP16 when half_table
    int half_table;
    uint32_t n_leaves;
    int storage;              // FPO_STORAGE_*
    int n1, n2, sig_stride, z_stride;  // strides in elements
    int stages;               // shared-memory pipeline depth (materialise_stages)
    int pipeline;             // 1: the frame-pipeline shape (materialise_pipeline_shape)
    int max_ctas_per_sm;      // 0: as many as fit
    int carveout;             // preferred shared-memory carveout in percent (0: the driver's default)
    double t, period_T;
    uint32_t *status;
    int test_timeout;         // 1: the first wait of each CTA gives up (failure-path test)
};

// Read-only view of a context's uploaded tree and launch settings.
struct CtxView {
    int device, sm_count;
    int n1, n2;
    double period_T;
    int traverse_threads, refill_min, inner_steps, max_steps;
    uint32_t *d_status;
    bool half_table;
    bool has_tree;
    uint32_t n_leaves, n_nodes, root_kind, n_smem_nodes;
    int depth;
    double aabb_min[3], aabb_size;
    const uint32_t *d_nodes, *d_perm;
    int storage;
    const void *d_sig, *d_z;
    const float *d_scale;
};
CtxView ctx_view(const fpo_ctx *ctx);
// Records `msg` as the calling thread's last error; returns `code`.
int set_last_error(int code, const char *msg);

// Argument checks shared by the render entry points (FPO_OK or the status
// they recorded): the rays (camera validity, finite t, ray count), and the
// options and output of one render.
int check_rays(const fpo_rays *r, uint64_t *n_rays);
int check_render_opts(const fpo_ctx *ctx, const fpo_frame_opts *opts, uint64_t n_rays, const float *out_rgb);
// Kernel parameters of one render (or adjoint) call; p.table is the context's
// own per-frame table, which a caller may point elsewhere.
TraverseParams traverse_params(const fpo_ctx *ctx, const fpo_rays *rays, const fpo_frame_opts *opts,
                               float *out_rgb, uint64_t n_rays);
// The per-frame table for time t into `table` on `stream`: the tensor-core
// decoder for LATENT storage, else the IDFT pass over the stored coefficients
// (at most max_ctas_per_sm CTAs per SM when > 0; with pipe_stages > 0 the
// frame-pipeline shape with that many stages and the given carveout).
// Returns a cudaError_t.
// test_timeout: the failure-path test of FPO_FLAG_TEST_DEVICE_TIMEOUT.
int launch_table_pass(const fpo_ctx *ctx, double t, float *table, int max_ctas_per_sm, void *stream,
                      int pipe_stages, int carveout, bool test_timeout);

// Latent decoder (per-leaf FP16 latents, MLP 32 -> 64 -> 64 -> n1 + 27 n2,
// ReLU).  Weights are BF16 bit patterns, row-major [out][in]; biases FP32.
struct LatentParams {
    const uint16_t *latents;  // FP16 [n_leaves][32]
    const uint16_t *w1;       // [64][32]
    const float *b1;          // [64]
    const uint16_t *w2;       // [64][64]
    const float *b2;          // [64]
    const uint16_t *w3;       // [n1 + 27 n2][64]
    const float *b3;          // [n1 + 27 n2]
    int n1, n2;
    double t, period_T;
    uint32_t n_leaves;
    float *table;             // [n_leaves][TABLE_STRIDE] FP32, or FP16 when half_table
    int half_table;
    uint32_t *status;
    int test_timeout;         // 1: each warpgroup's first wait gives up (failure-path test)
    int pipeline;             // 1: the frame-pipeline shape (one 256-thread CTA per SM)
    int carveout;             // preferred shared-memory carveout in percent (0: the driver's default)
    CUtensorMap table_map;    // set by launch_latent_table: the table as a [n_leaves][32] tensor
};

int launch_latent_table(const LatentParams &p, int sm_count, void *stream);
int latent_pipeline_smem_bytes();  // dynamic shared memory of the pipeline-shape decoder CTA

struct DecoderGradParams {
    fpo_mlp w, g;             // FP32 weights; gradients (accumulated)
    const uint32_t *rows;     // [batch] leaf rows (distinct)
    uint32_t batch;
    const float *latents;     // [N][32]
    const float *targets;     // [N][nc]
    const float *coef_weight; // [nc]
    const float *extra_dy;    // [N][nc] or nullptr
    float *dlatents;          // [batch][32]
    double *loss;             // accumulated, or nullptr
    int nc;
};
int launch_decoder_grad(const DecoderGradParams &p, int sm_count, void *stream);
int launch_gather_rows(const void *src, void *dst, const uint32_t *perm, uint32_t n, uint32_t bytes,
                       int sm_count, void *stream);
int decoder_grad_max_coeffs();
int launch_decoder_forward(const fpo_mlp &w, int nc, uint32_t n, const float *latents, float *out, int sm_count,
                           void *stream);
int launch_decode_records(const fpo_mlp &w, int n1, int n2, uint32_t n, const float *latents, const uint32_t *perm,
                          float *sig, float *zc, int sm_count, void *stream);
// The same on the tensor cores with the inference decoder's FP16 numerics
// (fpo_latent.cu); FP16-range and time-out reports go to *status.
int launch_decode_records_tc(const fpo_mlp &w, int n1, int n2, uint32_t n, const float *latents, const uint32_t *perm,
                             float *sig, float *zc, uint32_t *status, bool test_timeout, int sm_count, void *stream);
int launch_adam(float *param, const float *grad, float *m, float *v, uint64_t n, const uint32_t *rows, uint32_t dim,
                float lr, float b1, float b2, float eps, uint32_t step, int sm_count, void *stream);

struct BackwardParams {
    TraverseParams tp;          // rays, tree and options as for the fused forward
    const float *out_rgb;       // forward colour [rays][3]
    const float *dL_drgb;       // [rays][3]
    float *dL_dcoeffs;          // [n_leaves][n1 + 27 n2], canonical, upload order (accumulated)
    double *dL_dcoeffs64;       // the same in FP64 (gradient-check replay), else nullptr
    uint8_t *leaf_mark;         // optional [n_leaves] (upload order): set to 1 for every visited leaf
};

// Row-sparse Adam over the coefficients of the leaves a batch visited, fused
// with the write-back into the FP32 records and the reset of their gradient
// rows and marks.
struct LeafAdamParams {
    float *param, *grad, *m, *v;  // [n_leaves][nc], canonical, upload order
    uint8_t *leaf_mark;           // [n_leaves], upload order
    const uint32_t *perm;         // internal leaf -> upload id
    float *sig, *zc;              // FP32 records (internal order)
    uint32_t n_leaves;
    int n1, n2, sig_stride, z_stride;
    float lr, beta1, beta2, eps, bc1, bc2;  // bc = 1 - beta^step
};

// Launchers (return cudaError_t as int).
int launch_materialise(const MaterialiseParams &p, int sm_count, void *stream);
int materialise_stages(int storage, int n1, int n2);
// Shape of the IDFT pass when it shares each SM with the traversal (frame
// pipeline): CTAs per SM and stages such that the CTAs of one SM hold at most
// smem_budget bytes of records; smem_per_cta is the dynamic shared memory.
struct MatShape {
    int ctas_per_sm, stages, smem_per_cta;
};
MatShape materialise_pipeline_shape(int storage, int n1, int n2, int smem_budget);
int materialise_smem_bytes(const MaterialiseParams &p);  // dynamic shared memory of one CTA
int launch_backward(const BackwardParams &q, int sm_count, void *stream);
int launch_dft(const float *values, float *coeffs, uint32_t n_leaves, int n1, int n2, int T, uint32_t *status,
               bool test_timeout, int sm_count, void *stream);
int launch_set_coeffs(const float *src, const uint32_t *perm, float *sig, float *zc, uint32_t n_leaves,
                      int n1, int n2, int sm_count, void *stream);
int launch_leaf_adam(const LeafAdamParams &p, int sm_count, void *stream);
int launch_traverse(const TraverseParams &p, bool materialised, bool debug, int sm_count,
                    void *stream);
int traverse_smem_bytes(uint32_t n_smem_nodes, bool per_ray_basis, int threads);
bool fused_supported(int n1, int n2);

}  // namespace fpo
