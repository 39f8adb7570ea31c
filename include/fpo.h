/*
 * fpo.h - C ABI of the GB300 (sm_103a) Fourier PlenOctree renderer.
 *
 * Fourier PlenOctrees (Wang et al., "Fourier PlenOctrees for Dynamic Radiance
 * Field Rendering in Real-time", CVPR 2022) store, in every leaf of a union
 * octree (Sec. 4.2), n1 Fourier coefficients of the density and n2 Fourier
 * coefficients for each of the 3 (l_max+1)^2 SH colour coefficients
 * (Sec. 4.1, Eq. 6).  Rendering a frame at time t (the problem of Sec. 4.3:
 * the image of view i at frame t) evaluates the real inverse DFT of Eq. 7-9,
 * the SH colour of Eq. 1 with a sigmoid, and composites the exact ray-leaf
 * segments front to back (PlenOctree volume rendering, Sec. 3), stopping once
 * the transmittance falls below a threshold.
 *
 * Conventions for every call:
 *  - Return values are fpo_status codes; nothing throws across the ABI.
 *    fpo_last_error() gives a message for the last failure on this thread.
 *  - Pointers documented as "device" are CUDA device pointers owned by the
 *    caller; "host" pointers are read during the call only and may be freed
 *    afterwards.
 *  - Work is enqueued on the caller's CUDA stream (cudaStream_t passed as
 *    void *; NULL is the legacy default stream) and is asynchronous: outputs
 *    are valid once that stream has been synchronised.
 *  - Errors that only the device can see (a traversal step cap hit, a visit
 *    log too small) set a status word in the context; fpo_status_sync()
 *    reports and clears it.
 *  - Leaf ids at the boundary (visit logs, leaf marks, gradients) are the
 *    upload order of fpo_tree_desc, never internal addresses.
 *  - A context is not thread-safe: calls on one context must not overlap.
 *    Their GPU work shares the context's buffers (the per-frame table, the
 *    status word): enqueue it on one stream, or order the streams.
 */
#ifndef FPO_H
#define FPO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fpo_ctx fpo_ctx; /* opaque; owns the device copy of one tree */

typedef enum {
    FPO_OK = 0,
    FPO_ERR_INVALID_ARG = -1,     /* a NULL or out-of-range argument */
    FPO_ERR_OOM = -2,             /* device or host allocation failed */
    FPO_ERR_CUDA = -3,            /* a CUDA runtime call failed */
    FPO_ERR_BAD_TREE = -4,        /* leaves out of range, duplicated or nested */
    FPO_ERR_NO_TREE = -5,         /* render before fpo_upload_tree */
    FPO_ERR_TRAVERSAL_LIMIT = -6, /* device: a ray exceeded its step cap */
    FPO_ERR_VISIT_OVERFLOW = -7,  /* device: a ray had more visits than visit_cap */
    FPO_ERR_UNSUPPORTED = -8,     /* a valid request this build does not implement */
    FPO_ERR_DEVICE_TIMEOUT = -9,  /* device: a bounded wait on an async copy gave up */
    FPO_ERR_RANGE = -10           /* device: a latent decoder operand exceeded the FP16 range */
} fpo_status;

/* Storage precision of the leaf coefficients (the math is FP32 throughout). */
enum { FPO_STORAGE_F32 = 0, FPO_STORAGE_BF16 = 1, FPO_STORAGE_F16 = 2, FPO_STORAGE_FP8_E4M3 = 3,
       FPO_STORAGE_LATENT = 4 /* per-leaf FP16 latents + decoder (fpo_set_latents) */ };

/* Where the per-leaf inverse DFT (Eq. 7, Eq. 9) runs:
 *  FUSED        at every ray-leaf visit, from the stored coefficients;
 *  MATERIALISE  once per frame for every leaf (a 28-value table), which the
 *               traversal then reads;
 *  AUTO         the library's choice (currently MATERIALISE for camera frames,
 *               FUSED for rays with per-ray times). */
enum { FPO_IDFT_AUTO = 0, FPO_IDFT_FUSED = 1, FPO_IDFT_MATERIALISE = 2 };
/* Precision of the per-frame table of the MATERIALISE mode (sigma(t) and the
 * 27 z(t) of every leaf): FP32 (128 bytes per leaf) or FP16 (64 bytes per
 * leaf, half the table traffic of the traversal).  AUTO: FP32 with FP32
 * storage, FP16 with the reduced-precision and latent storages, whose
 * coefficients already carry fewer bits than FP16 keeps of sigma and z. */
enum { FPO_TABLE_AUTO = 0, FPO_TABLE_F32 = 1, FPO_TABLE_F16 = 2 };

typedef struct {
    int32_t n1;        /* density Fourier coefficients per leaf (paper: 31, Tab. 3) */
    int32_t n2;        /* Fourier coefficients per SH coefficient (paper: 5) */
    int32_t sh_degree; /* l_max (paper: 2, Sec. 5); only 2 is supported */
    double period_T;   /* T of Eq. 8: the sequence length in frames */
    int32_t storage;   /* FPO_STORAGE_* */
    int32_t idft_mode; /* FPO_IDFT_* */
    int32_t device;    /* CUDA device ordinal the context lives on */
    /* Launch tuning of the traversal (0 = library default): threads per CTA
     * (128 or 256); the number of idle lanes at which a warp refills them
     * with new rays (1..32; 32 refills only a fully idle warp); the number of
     * steps a lane takes between two such checks (default: to the end of its
     * ray). */
    int32_t traverse_threads;
    int32_t refill_min;
    int32_t inner_steps;
    int32_t table_precision; /* FPO_TABLE_* */
    /* Traversal steps a ray may take before it stops and the call reports
     * FPO_ERR_TRAVERSAL_LIMIT (0 = the library's bound 3 * 2^depth + 16,
     * which no ray of a valid tree reaches; a small value exercises the
     * device-side error path). */
    int32_t max_steps;
} fpo_config;

/* A union octree given by its leaves (Sec. 4.2): leaf j is the cell
 * leaf_xyz[j] (integer coordinates at level leaf_depth[j]) of the regular
 * 2^leaf_depth grid over the cube [aabb_min, aabb_min + aabb_size]^3.  Leaves
 * must be disjoint (no duplicates, no leaf inside another); anything not
 * covered by a leaf is empty space.  coeffs holds per leaf, in canonical
 * order, [k_sigma_0..k_sigma_{n1-1}] then [c=0..2][k=0..8][i=0..n2-1] with
 * k = l(l+1)+m, i.e. n1 + 27*n2 floats.  All arrays are host memory. */
typedef struct {
    uint32_t n_leaves;
    uint32_t max_depth; /* >= every leaf_depth; <= 12 */
    const uint8_t *leaf_depth;  /* [n_leaves] */
    const uint32_t *leaf_xyz;   /* [n_leaves][3] */
    const float *coeffs;        /* [n_leaves][n1 + 27*n2] */
    double aabb_min[3];
    double aabb_size;
} fpo_tree_desc;

enum { FPO_RAYS_CAMERA = 0, FPO_RAYS_EXPLICIT = 1 };

/* The rays of one render call.
 * CAMERA: a pinhole camera at `eye` looking at `target` with `up`, vertical
 *   field of view fov_y_deg, width x height pixels, row 0 at the top.  Pixel
 *   (px, py) shoots the unit ray through the pixel centre:
 *   d ~ f + sx r + sy u with f = |target - eye|, r = |f x up|, u = r x f,
 *   sx = (2 (px + 0.5)/W - 1) tan(fov/2) W/H, sy = (1 - 2 (py + 0.5)/H) tan(fov/2).
 *   Ray index = py * width + px.  All rays share the frame time t.
 * EXPLICIT: n rays with device arrays o[n][3], d[n][3] (d is normalised by
 *   the library; distances are measured along the unit direction) and an
 *   optional device array t_per_ray[n] (else every ray uses t). */
typedef struct {
    int32_t mode;
    double eye[3], target[3], up[3];
    double fov_y_deg;
    uint32_t width, height;
    double t;
    uint32_t n;
    const float *o, *d, *t_per_ray;
} fpo_rays;

enum {
    FPO_FLAG_RECORD_VISITS = 1, /* write visit_log / visit_count */
    FPO_FLAG_OUT_T = 2,         /* write the final transmittance to out_T */
    FPO_FLAG_MARK_LEAVES = 4,   /* set leaf_mark[id] = 1 for every visited leaf */
    FPO_FLAG_STATS = 8,         /* add traversal counters to stats[0..2] */
    /* Table mode, camera or explicit rays without per-ray times: if the
     * context's per-frame table was last built by fpo_render for the same t
     * (bit-equal) and nothing has changed the coefficients or latents since
     * (fpo_upload_tree, fpo_set_coeffs, fpo_adam_leaves, fpo_set_latents),
     * skip the IDFT pass and reuse it: several views of one frame time cost
     * one IDFT pass.  The call must follow the one that built the table on
     * the same stream (or an ordered one). */
    FPO_FLAG_REUSE_TABLE = 16,
    /* fpo_render_backward only: the gradient-check replay.  The FP32 stepping
     * still decides which leaves a ray visits, in which order and where it
     * stops (as in the forward); each visited leaf's segment is then measured
     * by an FP64 slab test of its box, and the IDFT, SH, sigmoid,
     * transmittance products and S_j run in FP64 over two replays of the ray
     * (the first accumulates the FP64 colour, so out_rgb is not used).
     * dL_dcoeffs then points to FP64 values (double [n_leaves][n1 + 27*n2],
     * 8-byte aligned).  Slow: for checking gradients, not for training. */
    FPO_FLAG_FP64_GRADCHECK = 32,
    /* Test of the device-side failure path (fpo_render in the table mode):
     * the first wait of every CTA of the table pass (the IDFT pass's wait
     * for its first bulk copies, or the latent decoder's wait for its first
     * MMAs) is made on a barrier that nothing signals, with a 1 ms limit.
     * The pass stops, waits (with its normal limit) for the copies or MMAs it
     * has in flight, and the call then reports FPO_ERR_DEVICE_TIMEOUT through
     * fpo_status_sync; the frame's pixels are undefined, and the context
     * renders normally afterwards.  (fpo_dft_leaves, fpo_decoder_grad_tc and
     * fpo_set_coeffs_from_decoder take it too, each as it documents.) */
    FPO_FLAG_TEST_DEVICE_TIMEOUT = 64,
    /* fpo_set_coeffs_from_decoder: decode on the tensor cores. */
    FPO_FLAG_TENSOR_CORES = 128
};

/* Per-call options.  bg: background colour added with the final
 * transmittance.  stop_T: early-stop threshold (the ray stops after the
 * first update that leaves T < stop_T; 0 disables).  Device outputs, each
 * used only when its flag is set: visit_log [rays][visit_cap] and
 * visit_count [rays] (leaf ids in visit order, count may exceed visit_cap,
 * which then also raises FPO_ERR_VISIT_OVERFLOW), out_T [rays], leaf_mark
 * [n_leaves] (never cleared by the library), stats [3] (device, accumulated:
 * traversal steps, leaf visits, rays that entered the tree).  events: optional cudaEvent_t
 * handles recorded on the stream before the first kernel of the frame,
 * between the IDFT pass and the traversal, and after the traversal. */
typedef struct {
    float bg[3];
    float stop_T;
    uint32_t flags;
    uint32_t *visit_log;
    uint32_t visit_cap;
    uint32_t *visit_count;
    float *out_T;
    uint8_t *leaf_mark;
    uint64_t *stats;
    void *events[3];
} fpo_frame_opts;

typedef struct {
    uint32_t n_leaves, n_nodes, max_depth, n_smem_nodes;
    uint64_t node_bytes;      /* device bytes of the node array */
    uint64_t leaf_bytes;      /* device bytes of the stored coefficients (or latents) */
    uint64_t leaf_record_bytes; /* stored bytes per leaf (padded); 64 for LATENT storage */
    uint64_t table_bytes;     /* device bytes of the per-frame IDFT table (0 until used) */
} fpo_tree_info;

/* Creates a context on cfg->device.  Validates n1 in [1, 32], n2 in [1, 16],
 * sh_degree == 2, period_T > 0, storage, idft_mode and tuning values.
 * Errors: INVALID_ARG, UNSUPPORTED, CUDA, OOM.  *out is NULL on failure. */
int fpo_create(fpo_ctx **out, const fpo_config *cfg);

/* Validates a tree description without any GPU (host only); the same checks
 * fpo_upload_tree runs.  Errors: INVALID_ARG, BAD_TREE. */
int fpo_validate_tree(const fpo_tree_desc *tree, const fpo_config *cfg);

/* Packs the union octree (Sec. 4.2) breadth-first and copies it and the leaf
 * coefficients (Sec. 4.1, Eq. 6) to the device, replacing any previous tree.
 * Blocks until the copies are done.  Errors: INVALID_ARG, BAD_TREE, OOM, CUDA. */
int fpo_upload_tree(fpo_ctx *ctx, const fpo_tree_desc *tree);

/* Renders the rays at frame time t (Sec. 4.1, Eq. 7-9 and Eq. 1; compositing
 * as in Sec. 3) into out_rgb, a device array [rays][3] of FP32 RGB.
 * Zero rays is valid and launches nothing.  Errors (synchronous): NO_TREE,
 * INVALID_ARG, CUDA.  Device-side errors: see fpo_status_sync. */
int fpo_render(fpo_ctx *ctx, const fpo_rays *rays, const fpo_frame_opts *opts,
               float *out_rgb, void *cuda_stream);

/* Renders a sequence of frames (e.g. the frames of a free-viewpoint video)
 * into out_rgb, device [n_frames][rays][3]; every frame has the same number
 * of rays (camera or explicit rays without per-ray times) and the same
 * options, which carry no debug outputs (flags must be 0; opts->events are
 * ignored).  frame_done: NULL, or host array [n_frames] of cudaEvent_t
 * handles (NULL entries allowed); event k is recorded once frame k's pixels
 * are written (on the stream that traversed it), so a caller can read frame
 * k back while later frames render.  The result equals n_frames calls of
 * fpo_render.  In the table mode the work is pipelined over four slots:
 * frame k uses slot k mod 4, with its own table (the context keeps four:
 * 4 x n_leaves x 128 bytes, 64 for an FP16 table), traversal stream (slot 0:
 * cuda_stream; the others internal) and tile counter; the tables of the
 * next frames are computed on another internal stream while earlier frames
 * are traversed (frames that all share one t, bit-equal, take a single
 * table pass), and consecutive traversals may overlap (the call orders
 * all of it after cuda_stream's previous work and before everything
 * enqueued on cuda_stream after the call).  Both kernels
 * share every SM: the call picks their launch shapes itself (two 384-thread
 * traversal CTAs and one or two IDFT CTAs per SM, or for LATENT storage one
 * 256-thread decoder CTA, with a shared-memory carveout that holds them
 * all), whatever traverse_threads says.  Errors: as fpo_render. */
int fpo_render_frames(fpo_ctx *ctx, const fpo_rays *frames, uint32_t n_frames,
                      const fpo_frame_opts *opts, float *out_rgb, void *const *frame_done,
                      void *cuda_stream);

/* Adjoint of fpo_render (the back-propagation of Sec. 4.3, used to fine-tune
 * the leaf coefficients against the loss of Eq. 13): given dL/d(rgb) (device
 * [rays][3]) it accumulates dL/d(coefficients) into dL_dcoeffs, a device
 * array [n_leaves][n1 + 27*n2] in canonical order and upload order (the
 * caller zeroes it; 16-byte aligned, as cudaMalloc returns it).  out_rgb is the forward colour of the same rays and
 * options.  Each ray is replayed with the per-visit IDFT, so the segments and
 * the early stop are those of a FUSED-mode forward (treated as fixed: the
 * truncation is part of the function); sigma = max(0, sigma_raw) passes no
 * gradient where sigma_raw <= 0.  Needs FP32 storage and (n1, n2) in
 * {(31,5), (11,5), (21,5), (31,11)}; otherwise FPO_ERR_UNSUPPORTED.
 * Of the debug flags only FPO_FLAG_MARK_LEAVES is honoured: it sets
 * leaf_mark[id] = 1 for every leaf the replay visits (the rows that receive
 * gradient), which fpo_adam_leaves consumes; the others are ignored.
 * FPO_FLAG_FP64_GRADCHECK selects the FP64 replay (see the flag).
 * Errors: INVALID_ARG, NO_TREE, UNSUPPORTED, CUDA. */
int fpo_render_backward(fpo_ctx *ctx, const fpo_rays *rays, const fpo_frame_opts *opts,
                        const float *out_rgb, const float *dL_drgb, float *dL_dcoeffs,
                        void *cuda_stream);

/* Renders like fpo_render in the MATERIALISE mode, but allocates nothing.
 * The paper has no counterpart: this entry point serves callers that cannot
 * call cudaMalloc when they render (for example a host framework that owns
 * all device memory through its own allocator, or a real-time loop that
 * forbids allocation after start-up).  fpo_render allocates the per-frame
 * IDFT table on first use; this call instead keeps it in a fixed array of
 * device memory inside the library: 8 MiB, loaded on every GPU that loads
 * the library and held until the process exits, enough for trees of at most
 * 65536 leaves.  Larger trees, and explicit rays with per-ray times, are
 * rejected with FPO_ERR_INVALID_ARG; LATENT storage with
 * FPO_ERR_UNSUPPORTED.  Inputs: ctx (a context whose tree was uploaded
 * beforehand) and rays; output: out_rgb as in fpo_render; opts and
 * device-side errors as in fpo_render (read them with fpo_status_sync).
 * The array is shared by all calls on a device and keeps the last call's
 * table: calls whose GPU work overlaps (different streams, or different
 * contexts on the same device) race on it and must be ordered.  The first
 * call on each device looks up the array's device address (once, under a
 * lock); make that first call before any stream capture begins. */
int fpo_render_noalloc(fpo_ctx *ctx, const fpo_rays *rays, const fpo_frame_opts *opts,
                       float *out_rgb, void *cuda_stream);

/* Replaces the coefficients of the uploaded tree with `coeffs`, a device
 * array [n_leaves][n1 + 27*n2] in canonical order and upload order (the
 * in-place update of the fine-tuning stage, Sec. 4.3).  Enqueued on the
 * stream.  Needs FP32 storage (else FPO_ERR_UNSUPPORTED).
 * Errors: INVALID_ARG, NO_TREE, UNSUPPORTED, CUDA. */
int fpo_set_coeffs(fpo_ctx *ctx, const float *coeffs, void *cuda_stream);

/* One optimiser step of the fine-tuning stage (Sec. 4.3, loss of Eq. 13)
 * on the leaves a batch visited: Adam (Kingma & Ba; lr, beta1, beta2, eps,
 * step >= 1 for the bias corrections 1 - beta^step) on every row of param
 * whose leaf_mark is non-zero, using the gradient row of grad (as
 * accumulated by fpo_render_backward with FPO_FLAG_MARK_LEAVES), with the
 * moment rows m and v (zero before the first step).  Rows without a mark are
 * left alone, as in a sparse-gradient Adam.  For each updated leaf the new
 * coefficients also go into the context's FP32 records (what fpo_set_coeffs
 * would write), and its grad row and mark are reset to zero, ready for the
 * next batch.  param, grad, m, v: device [n_leaves][n1 + 27*n2], canonical
 * order and upload order, caller-owned; leaf_mark: device [n_leaves].
 * Enqueued on the stream.  Needs FP32 storage (else FPO_ERR_UNSUPPORTED).
 * Errors: INVALID_ARG, NO_TREE, UNSUPPORTED, CUDA. */
int fpo_adam_leaves(fpo_ctx *ctx, float *param, float *grad, float *m, float *v, uint8_t *leaf_mark,
                    float lr, float beta1, float beta2, float eps, uint32_t step, void *cuda_stream);

/* Per-leaf DFT of the Fourier PlenOctree generation (Sec. 4.2, Eq. 10-12):
 * from the values every leaf of the unified octree takes at frames
 * t = 1..n_frames (device [n_frames][n_leaves][28]: sigma, then z_{c,k} for
 * c = 0..2, k = 0..8), computes the coefficients (device [n_leaves][n1 +
 * 27*n2], canonical order) k_i = sum_t x(t) (w_i / T) {cos(i pi t / T) for
 * even i, sin((i+1) pi t / T) for odd i} with T = n_frames, w_0 = 1 and
 * w_i = 2 for i >= 1, so that Eq. 8 inverts it exactly for signals of
 * frequency below T/2 (the paper prints w_i = 1, under which Eq. 8 would
 * halve every non-constant term).  Runs on the current device and stream.
 * With n2 = 5 and a 16-byte aligned `values`, frames are moved by bulk
 * asynchronous copies whose waits are bounded: a copy that has not landed
 * after 2 s makes its CTA write NaN to every coefficient of its unfinished
 * tiles, wait (bounded) for its copies in flight, and OR the value 4 (a
 * device-side wait gave up: FPO_ERR_DEVICE_TIMEOUT) into *status.  status: an optional
 * device word (NULL: the NaN coefficients alone show it); flags: 0, or
 * FPO_FLAG_TEST_DEVICE_TIMEOUT to make each CTA's first wait run out after
 * 1 ms (tests of that path).
 * Errors: INVALID_ARG (n1 in [1, 32], n2 in [1, 16], n_frames in [1, 256],
 * unknown flags), CUDA. */
int fpo_dft_leaves(int32_t n1, int32_t n2, uint32_t n_frames, uint32_t n_leaves,
                   const float *values, float *coeffs, uint32_t *status, uint32_t flags, void *cuda_stream);

/* One frame's octree for fpo_union_trees (host arrays): leaves as in
 * fpo_tree_desc, values [n_leaves][28] = sigma, then z_{c,k} (c = 0..2,
 * k = 0..8) of each leaf at that frame. */
typedef struct {
    uint32_t n_leaves;
    const uint8_t *leaf_depth;
    const uint32_t *leaf_xyz;
    const float *values;
} fpo_frame_tree;

/* Union of the frames' octree structures (Sec. 4.2): a cell is divided in the
 * union if any frame divides it, so every union leaf is as deep as or deeper
 * than the frame leaves holding it; a frame's value is copied into every
 * union leaf its (coarser) leaf was divided into, and is zero where that
 * frame has no leaf.  Host only.  Call with capacity 0 to learn *n_union;
 * then with host arrays union_depth [capacity], union_xyz [capacity][3] and
 * union_values [n_frames][capacity][28] (pass capacity = n_union for a dense
 * array).  Union leaves come in depth-first octant order (x, then y, then z
 * bit), i.e. Morton order.  Errors: INVALID_ARG, BAD_TREE (a frame's leaves
 * overlap or leave their grid). */
int fpo_union_trees(uint32_t n_frames, const fpo_frame_tree *frames, uint32_t max_depth,
                    uint32_t *n_union, uint8_t *union_depth, uint32_t *union_xyz,
                    float *union_values, uint32_t capacity);

/* A latent decoder: per leaf a 32-dim FP16 latent, decoded by a shared MLP
 * 32 -> 64 -> 64 -> n1 + 27*n2 with ReLU after the first two layers (the
 * learned stand-in for the per-leaf coefficients of Sec. 4.1; the paper's own
 * network Phi of Eq. 6 maps positions to coefficients).  Device arrays:
 * weights as BF16 bit patterns, row-major [out][in]; biases FP32. */
typedef struct {
    const uint16_t *w1; /* [64][32] */
    const float *b1;    /* [64] */
    const uint16_t *w2; /* [64][64] */
    const float *b2;    /* [64] */
    const uint16_t *w3; /* [n1 + 27*n2][64] */
    const float *b3;    /* [n1 + 27*n2] */
} fpo_decoder;

/* The per-frame table of fpo_render's MATERIALISE mode, decoded from
 * latents on the tensor cores: for every leaf, [max(0, sigma(t)), z_{c,k}(t)
 * x 27, 0 x 4] (device [n_leaves][32] FP32) where the coefficients are the
 * decoder's output and sigma, z follow Eq. 7 and Eq. 9 at time t.  The IDFT
 * is folded into the last layer (W3' = B(t) W3), so the MLP runs 32 -> 64 ->
 * 64 -> 28 with FP16 operands and FP32 accumulation (BF16 weights are
 * converted to FP16 in shared memory: FP16 keeps 3 more significant bits
 * than BF16, in a range of +-65504).  latents: device FP16 [n_leaves][32],
 * 16-byte aligned.
 * status: optional device word that receives the bit of
 * FPO_ERR_DEVICE_TIMEOUT when a bounded wait gives up, and that of
 * FPO_ERR_RANGE when a weight, bias or hidden activation is beyond the FP16
 * range (the table is then wrong).  Runs on the current device and stream.
 * Errors: INVALID_ARG, CUDA. */
int fpo_latent_table(const fpo_decoder *dec, int32_t n1, int32_t n2, double t, double period_T,
                     uint32_t n_leaves, const uint16_t *latents, float *table, uint32_t *status,
                     void *cuda_stream);

/* FP32 master weights of the latent decoder (device, shapes as fpo_decoder). */
typedef struct {
    float *w1, *b1, *w2, *b2, *w3, *b3;
} fpo_mlp;

/* One gradient evaluation for training the latent decoder: for the leaves
 * `rows` (device [batch], distinct), decodes y = MLP(latents[row]) in FP32 and
 * accumulates, for L = sum_rows sum_j coef_weight[j] (y_j - targets[row][j])^2
 * (+ sum extra_dy . y when extra_dy, device [N][n1+27*n2], is given, e.g. the
 * render adjoint's dL/d(coefficients)), the weight gradients into `grad`
 * (the caller zeroes them), writes dL/d(latent) of each batch row to
 * dlatents (device [batch][32]) and adds L to *loss (device, optional).
 * latents [N][32] and targets [N][n1+27*n2] are device FP32.
 * Errors: INVALID_ARG, CUDA. */
int fpo_decoder_grad(const fpo_mlp *w, int32_t n1, int32_t n2, uint32_t batch, const uint32_t *rows,
                     const float *latents, const float *targets, const float *coef_weight,
                     const float *extra_dy, const fpo_mlp *grad, float *dlatents, double *loss,
                     void *cuda_stream);

/* fpo_decoder_grad on the tensor cores (tcgen05, BF16 operands, FP32
 * accumulation in TMEM): the same loss, gradients and outputs, with every
 * matrix product of the forward pass and of the back-propagation taken
 * with BF16 operands (latents, weights, activations and dL/dy rounded to
 * BF16; each bias carried to about 16 bits as a BF16 pair), so results
 * agree with fpo_decoder_grad to the BF16 rounding of those operands.
 * status: an optional device word that a wait for the tensor cores which
 * runs out (2 s) ORs the value 4 into (FPO_ERR_DEVICE_TIMEOUT; the weight
 * gradients are then left unchanged); flags: 0, or
 * FPO_FLAG_TEST_DEVICE_TIMEOUT to make each CTA's first wait run out after
 * 1 ms (tests of that path).  One CTA per SM holds all 512 TMEM columns.
 * Errors: INVALID_ARG, CUDA. */
int fpo_decoder_grad_tc(const fpo_mlp *w, int32_t n1, int32_t n2, uint32_t batch, const uint32_t *rows,
                        const float *latents, const float *targets, const float *coef_weight,
                        const float *extra_dy, const fpo_mlp *grad, float *dlatents, double *loss,
                        uint32_t *status, uint32_t flags, void *cuda_stream);

/* The decoded coefficients of n leaves in FP32: coeffs[i] = MLP(latents[i])
 * (device [n][32] in, device [n][n1 + 27*n2] out, canonical order), with the
 * FP32 master weights.  Used to put the decoder's current coefficients into
 * an FP32 context (fpo_set_coeffs), e.g. for the render adjoint of a pixel
 * loss while the decoder trains.  Runs on the current device and stream.
 * Errors: INVALID_ARG, CUDA. */
int fpo_decoder_forward(const fpo_mlp *w, int32_t n1, int32_t n2, uint32_t n, const float *latents,
                        float *coeffs, void *cuda_stream);

/* fpo_set_coeffs of the decoder's coefficients: every leaf's latent
 * (latents: device [n_leaves][32], upload order) decoded by the MLP `w`
 * (FP32 master weights) straight into the context's FP32 records, with no
 * [n_leaves][n1 + 27*n2] array in between.  flags = 0: in FP32, the values
 * fpo_decoder_forward followed by fpo_set_coeffs writes (the same
 * arithmetic, bit for bit).  FPO_FLAG_TENSOR_CORES: on the tensor cores with
 * the inference decoder's numerics (FP16 latents, weights and hidden
 * activations, FP32 accumulation; the last layer unfolded): what the LATENT
 * storage would render before the IDFT folding; an operand beyond the FP16
 * range or a wait that runs out (2 s; 1 ms for the first with
 * FPO_FLAG_TEST_DEVICE_TIMEOUT) is reported through fpo_status_sync as
 * FPO_ERR_RANGE / FPO_ERR_DEVICE_TIMEOUT.  Enqueued on the stream.  Needs
 * FP32 storage and n1 + 27*n2 <= 176 (else FPO_ERR_UNSUPPORTED).
 * Errors: INVALID_ARG (including unknown flags), NO_TREE, UNSUPPORTED, CUDA. */
int fpo_set_coeffs_from_decoder(fpo_ctx *ctx, const fpo_mlp *w, const float *latents, uint32_t flags,
                                void *cuda_stream);

/* Adam step (Kingma & Ba 2015) with bias correction, step counted from 1:
 * dense over n elements (rows NULL), or over the rows of a batch (device
 * rows [n / dim], distinct; param, m, v [N][dim]; grad [n / dim][dim]).
 * Errors: INVALID_ARG, CUDA. */
int fpo_adam(float *param, const float *grad, float *m, float *v, uint64_t n, const uint32_t *rows,
             uint32_t dim, float lr, float beta1, float beta2, float eps, uint32_t step,
             void *cuda_stream);

/* LATENT storage: gives the uploaded tree its per-leaf latents (device FP16
 * [n_leaves][32], upload order) and decoder (device arrays, copied into the
 * context).  fpo_render then decodes the per-frame table with
 * fpo_latent_table's tensor-core kernel before the traversal.  The tree is
 * uploaded with coeffs = NULL for this storage.  Enqueued on the stream.
 * Errors: INVALID_ARG, NO_TREE, UNSUPPORTED (context storage is not LATENT), OOM, CUDA. */
int fpo_set_latents(fpo_ctx *ctx, const uint16_t *latents, const fpo_decoder *dec, void *cuda_stream);

/* Waits for cuda_stream and returns (then clears) the device status word:
 * FPO_OK, FPO_ERR_TRAVERSAL_LIMIT, FPO_ERR_VISIT_OVERFLOW,
 * FPO_ERR_DEVICE_TIMEOUT or FPO_ERR_RANGE. */
int fpo_status_sync(fpo_ctx *ctx, void *cuda_stream);

/* Sizes of the uploaded tree.  Errors: INVALID_ARG, NO_TREE. */
int fpo_tree_info_get(const fpo_ctx *ctx, fpo_tree_info *out);

/* Releases every device and host allocation of the context.  NULL-safe. */
void fpo_destroy(fpo_ctx *ctx);

/* Message of the last failure on the calling thread ("" if none). */
const char *fpo_last_error(void);

/* Diagnostics.  FP32 FMA throughput microbenchmark: `blocks` x `threads`
 * threads (threads a multiple of 32, at most 1024) each run 16 independent
 * chains of `iters` fused multiply-adds and store one float into sink
 * (device, blocks * threads floats, caller-owned); *flops (host, optional)
 * receives the floating-point operations the launch performs (2 per FMA).
 * Time it with events on the stream: flops / seconds is the device's FP32
 * FMA rate, the roofline denominator of the SIMT arithmetic kernels.
 * Errors: INVALID_ARG, CUDA. */
int fpo_fma_peak(uint32_t blocks, uint32_t threads, uint32_t iters, float *sink, double *flops, void *cuda_stream);

/* ABI version: 100 * major + minor (1.1: fpo_render_frames takes frame_done;
 * 1.2: fpo_set_coeffs_from_decoder, fpo_decoder_grad_tc, fpo_fma_peak; fpo_dft_leaves takes
 * status and flags). */
int fpo_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FPO_H */
