// CUDA kernels of the FPO renderer (sm_103a).
//
//  materialise_kernel   per-frame inverse DFT of every leaf (Eq. 7, Eq. 9):
//                       n1 + 27 n2 stored coefficients -> a 32-float record
//                       [sigma(t) >= 0, z_{c,k}(t) x 27, 0 x 4].
//  traverse_kernel      persistent ray traversal of the union octree with
//                       exact ray-leaf segments and empty-space skipping,
//                       SH colour + sigmoid (Eq. 1) and front-to-back
//                       compositing with early stop; the IDFT either read
//                       from the per-frame table or fused per visit.
#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>

#include "fpo_internal.h"

namespace fpo {
namespace {

constexpr int TRAV_THREADS = 256;   // 8 warps; each warp traces 8x4-pixel tiles
constexpr int STACK_LEVELS = MAX_DEPTH + 1;
constexpr int MAX_BASIS = 64;

// Real SH of degree <= 2 at a unit direction, index k = l(l+1)+m
// (orthonormal; sign convention of the complex SH with Condon-Shortley phase).
__device__ __forceinline__ void sh_basis(float x, float y, float z, float Y[9])
{
    const float c0 = 0.28209479177387814f;   // 1/(2 sqrt(pi))
    const float c1 = 0.48860251190291992f;   // sqrt(3/(4 pi))
    const float c2 = 1.09254843059207907f;   // sqrt(15/pi)/2
    const float c3 = 0.31539156525252005f;   // sqrt(5/pi)/4
    const float c4 = 0.54627421529603959f;   // sqrt(15/pi)/4
    Y[0] = c0;
    Y[1] = -c1 * y;
    Y[2] = c1 * z;
    Y[3] = -c1 * x;
    Y[4] = c2 * x * y;
    Y[5] = -c2 * y * z;
    Y[6] = c3 * (3.0f * z * z - 1.0f);
    Y[7] = -c2 * x * z;
    Y[8] = c4 * (x * x - y * y);
}

// Eq. 8 at one time, computed in FP64 (cospi/sinpi of i t / T) and rounded.
__device__ __forceinline__ float basis_fp64(int i, double t, double period)
{
    const double u = t / period;
    return (i & 1) ? (float)sinpi((double)(i + 1) * u) : (float)cospi((double)i * u);
}

// Eq. 8 from an FP32 time (explicit rays with per-ray times).
__device__ __forceinline__ float basis_fp32(int i, float u /* t / T */)
{
    const float a = (float)((i & 1) ? (i + 1) : i) * u;
    const float r = a - 2.0f * floorf(0.5f * a);  // reduce mod 2 (period of cospi)
    return (i & 1) ? sinpif(r) : cospif(r);
}

__device__ __forceinline__ float sigmoidf_(float x) { return 1.0f / (1.0f + __expf(-x)); }

}  // namespace

// ---------------------------------------------------------------------------
// Per-frame IDFT table.  One warp per leaf: lanes 1..27 each form one
// z_{c,k}(t) from n2 coefficients (coalesced: consecutive lanes read
// consecutive n2-float groups), lanes 28..31 form partial density sums over
// 8-term slices, reduced by shuffles into lane 0.

__global__ void __launch_bounds__(256) materialise_kernel(const __grid_constant__ MaterialiseParams p)
{
    __shared__ float s_b[MAX_BASIS];
    const int nb = p.n1 > p.n2 ? p.n1 : p.n2;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s_b[i] = basis_fp64(i, p.t, p.period_T);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    float bz[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) bz[i] = i < p.n2 ? s_b[i] : 0.0f;
    for (uint32_t leaf = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; leaf < p.n_leaves;
         leaf += warps) {
        float v = 0.0f;
        if (lane >= 1 && lane <= 27) {
            const float *z = p.zc + (size_t)leaf * p.z_stride + (lane - 1) * p.n2;
            for (int i = 0; i < p.n2; ++i) v = fmaf(__ldg(z + i), bz[i], v);
        } else if (lane >= 28) {
            const float *s = p.sig + (size_t)leaf * p.sig_stride;
            const int i0 = (lane - 28) * 16;
            for (int i = i0; i < i0 + 16 && i < p.n1; ++i) v = fmaf(__ldg(s + i), s_b[i], v);
        }
        float part = lane >= 28 ? v : 0.0f;
        part += __shfl_xor_sync(0xffffffffu, part, 1);
        part += __shfl_xor_sync(0xffffffffu, part, 2);
        const float sig = __shfl_sync(0xffffffffu, part, 28);
        float outv = lane == 0 ? fmaxf(sig, 0.0f) : (lane <= 27 ? v : 0.0f);
        p.table[(size_t)leaf * TABLE_STRIDE + lane] = outv;
    }
}

int launch_materialise(const MaterialiseParams &p, int sm_count, void *stream)
{
    if (p.n_leaves == 0) return (int)cudaSuccess;
    const int threads = 256;
    uint64_t want = ((uint64_t)p.n_leaves * 32 + threads - 1) / threads;
    uint64_t cap = (uint64_t)sm_count * 8;
    int blocks = (int)(want < cap ? want : cap);
    materialise_kernel<<<blocks, threads, 0, (cudaStream_t)stream>>>(p);
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Traversal.

namespace {

struct FrameShared {
    float b[MAX_BASIS];
    float f[3], r[3], u[3], eye[3];
    float sx_scale, sy_scale;
};

template <bool MAT, bool DBG, int N1, int N2>
__device__ void trace_ray(const TraverseParams &p, const FrameShared &fs,
                          const uint32_t *__restrict__ s_nodes, uint32_t *s_stack, int stride,
                          uint32_t ray, int px, int py)
{
    // --- ray generation (camera mode) or load (explicit rays) --------------
    float ox, oy, oz, dx, dy, dz;
    constexpr int NB = N1 > N2 ? N1 : N2;
    float b[NB > 0 ? NB : 1];
    const bool own_basis = !MAT && p.fr.mode == FPO_RAYS_EXPLICIT && p.fr.rt != nullptr;
    if (p.fr.mode == FPO_RAYS_CAMERA) {
        const float sx = (2.0f * ((float)px + 0.5f) / (float)p.fr.width - 1.0f) * fs.sx_scale;
        const float sy = (1.0f - 2.0f * ((float)py + 0.5f) / (float)p.fr.height) * fs.sy_scale;
        dx = fs.f[0] + sx * fs.r[0] + sy * fs.u[0];
        dy = fs.f[1] + sx * fs.r[1] + sy * fs.u[1];
        dz = fs.f[2] + sx * fs.r[2] + sy * fs.u[2];
        ox = fs.eye[0];
        oy = fs.eye[1];
        oz = fs.eye[2];
    } else {
        ox = p.fr.ro[3 * ray];
        oy = p.fr.ro[3 * ray + 1];
        oz = p.fr.ro[3 * ray + 2];
        dx = p.fr.rd[3 * ray];
        dy = p.fr.rd[3 * ray + 1];
        dz = p.fr.rd[3 * ray + 2];
    }
    {
        const float inv = 1.0f / sqrtf(dx * dx + dy * dy + dz * dz);
        dx *= inv;
        dy *= inv;
        dz *= inv;
    }
    if (!MAT) {
        if (own_basis) {
            const float u = p.fr.rt[ray] / (float)p.fr.period_T;
#pragma unroll
            for (int i = 0; i < NB; ++i) b[i] = basis_fp32(i, u);
        } else {
#pragma unroll
            for (int i = 0; i < NB; ++i) b[i] = fs.b[i];
        }
    }
    float Y[9];
    sh_basis(dx, dy, dz, Y);

    float C0 = 0.0f, C1 = 0.0f, C2 = 0.0f, T = 1.0f;
    uint32_t n_visits = 0;

    // --- clip against the grid [0, G]^3 in grid units ---------------------
    const int D = p.depth;
    const int G = 1 << D;
    const float gs = p.grid_scale;
    float go[3] = {(ox - p.amin[0]) * gs, (oy - p.amin[1]) * gs, (oz - p.amin[2]) * gs};
    const float gd[3] = {dx * gs, dy * gs, dz * gs};
    float inv[3];
    float t0 = 0.0f, t1 = FLT_MAX;
    bool hit = p.root_kind != ROOT_EMPTY;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (gd[a] != 0.0f) {
            inv[a] = 1.0f / gd[a];
            const float ta = (0.0f - go[a]) * inv[a], tb = ((float)G - go[a]) * inv[a];
            t0 = fmaxf(t0, fminf(ta, tb));
            t1 = fminf(t1, fmaxf(ta, tb));
        } else {
            inv[a] = 0.0f;
            if (go[a] < 0.0f || go[a] > (float)G) hit = false;
        }
    }
    hit = hit && (t0 < t1);

    if (hit) {
        // Work relative to the entry point: t measured from there.
#pragma unroll
        for (int a = 0; a < 3; ++a) go[a] = fmaf(t0, gd[a], go[a]);
        int P[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) P[a] = min(max((int)floorf(go[a]), 0), G - 1);

        float t = 0.0f;
        uint32_t steps = 0;
        int lvl_start = 0;  // deepest ancestor level still valid in the stack
        uint32_t node = 0;
        if (p.root_kind == ROOT_NODE) s_stack[0] = 0;
        for (;;) {
            // --- locate the cube containing P -----------------------------
            int lvl = lvl_start;
            uint32_t kind, leaf = 0;
            if (p.root_kind == ROOT_LEAF) {
                lvl = 0;
                kind = ROOT_LEAF;
            } else {
                node = s_stack[lvl * stride];
                for (;;) {
                    const int sh = D - 1 - lvl;
                    const uint32_t c = ((P[0] >> sh) & 1) | (((P[1] >> sh) & 1) << 1) |
                                       (((P[2] >> sh) & 1) << 2);
                    const uint32_t idx = node * 8 + c;
                    const uint32_t s = idx < p.n_smem_nodes * 8 ? s_nodes[idx] : __ldg(p.nodes + idx);
                    ++lvl;
                    if (s == 0u) { kind = ROOT_EMPTY; break; }
                    if (s & LEAF_BIT) { kind = ROOT_LEAF; leaf = s & ~LEAF_BIT; break; }
                    node = s;
                    s_stack[lvl * stride] = node;
                }
            }
            // --- exit of the cube: level lvl, size 2^(D - lvl) cells -------
            const int csz = 1 << (D - lvl);
            float te[3];
            int lo[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                lo[a] = P[a] & ~(csz - 1);
                if (gd[a] > 0.0f)
                    te[a] = ((float)(lo[a] + csz) - go[a]) * inv[a];
                else if (gd[a] < 0.0f)
                    te[a] = ((float)lo[a] - go[a]) * inv[a];
                else
                    te[a] = FLT_MAX;
            }
            int m = 0;
            float tx = te[0];
            if (te[1] < tx) { tx = te[1]; m = 1; }
            if (te[2] < tx) { tx = te[2]; m = 2; }

            // --- shade a leaf segment ------------------------------------
            if (kind == ROOT_LEAF && tx > t) {
                const float delta = tx - t;
                float sigma, z[27];
                if (MAT) {
                    const float4 *rec = p.table + (size_t)leaf * (TABLE_STRIDE / 4);
                    float v[28];
#pragma unroll
                    for (int q = 0; q < 7; ++q) {
                        const float4 w = __ldg(rec + q);
                        v[4 * q] = w.x;
                        v[4 * q + 1] = w.y;
                        v[4 * q + 2] = w.z;
                        v[4 * q + 3] = w.w;
                    }
                    sigma = v[0];
#pragma unroll
                    for (int q = 0; q < 27; ++q) z[q] = v[q + 1];
                } else {
                    // Eq. 7 then Eq. 9 at this visit, from the stored records.
                    const float4 *sr = p.sig + (size_t)leaf * p.sig_stride4;
                    float acc = 0.0f;
#pragma unroll
                    for (int q = 0; q < (N1 + 3) / 4; ++q) {
                        const float4 w = __ldg(sr + q);
                        const float wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            if (4 * q + j < N1) acc = fmaf(wv[j], b[4 * q + j], acc);
                    }
                    sigma = fmaxf(acc, 0.0f);
                    const float4 *zr = reinterpret_cast<const float4 *>(p.zc + (size_t)leaf * p.z_stride);
#pragma unroll
                    for (int q = 0; q < 27; ++q) z[q] = 0.0f;
#pragma unroll
                    for (int q4 = 0; q4 < (27 * N2 + 3) / 4; ++q4) {
                        const float4 w = __ldg(zr + q4);
                        const float wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int e = 4 * q4 + j;
                            if (e < 27 * N2) z[e / N2] = fmaf(wv[j], b[e % N2], z[e / N2]);
                        }
                    }
                }
                float col[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float s = 0.0f;
#pragma unroll
                    for (int k = 0; k < 9; ++k) s = fmaf(z[9 * c + k], Y[k], s);
                    col[c] = sigmoidf_(s);
                }
                const float e = __expf(-sigma * delta);
                const float w = T * (1.0f - e);
                C0 = fmaf(w, col[0], C0);
                C1 = fmaf(w, col[1], C1);
                C2 = fmaf(w, col[2], C2);
                T *= e;
                if (DBG) {
                    if (p.flags & FPO_FLAG_RECORD_VISITS) {
                        if (n_visits < p.visit_cap)
                            p.visit_log[(size_t)ray * p.visit_cap + n_visits] = p.perm[leaf];
                        else
                            atomicOr(p.status, STATUS_VISIT_OVERFLOW);
                    }
                    if (p.flags & FPO_FLAG_MARK_LEAVES) p.leaf_mark[p.perm[leaf]] = 1;
                }
                ++n_visits;
                if (T < p.stop_T) break;
            }
            // --- step into the neighbour cube ----------------------------
            // Along m: the adjacent cube; along the other axes: the cell
            // holding the exit point, clamped to this cube's extent and never
            // moving backwards (so every step makes progress).
            int Pn[3];
            bool inside = true;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (a == m) {
                    Pn[a] = gd[a] > 0.0f ? lo[a] + csz : lo[a] - 1;
                    inside = Pn[a] >= 0 && Pn[a] < G;
                } else {
                    int q = (int)floorf(fmaf(tx, gd[a], go[a]));
                    q = min(max(q, lo[a]), lo[a] + csz - 1);
                    if (gd[a] > 0.0f) q = max(q, P[a]);
                    else if (gd[a] < 0.0f) q = min(q, P[a]);
                    Pn[a] = q;
                }
            }
            if (!inside) break;
            t = fmaxf(t, tx);
            // deepest common ancestor of the old and the new cell
            const uint32_t diff = (uint32_t)((P[0] ^ Pn[0]) | (P[1] ^ Pn[1]) | (P[2] ^ Pn[2]));
            const int hb = 31 - __clz(diff);  // diff != 0: P moved along m
            lvl_start = D - 1 - hb;
            P[0] = Pn[0];
            P[1] = Pn[1];
            P[2] = Pn[2];
            if (++steps > p.max_steps) {
                atomicOr(p.status, STATUS_TRAVERSAL_LIMIT);
                break;
            }
        }
    }
    const float bgw = T;
    p.out_rgb[3 * (size_t)ray] = fmaf(bgw, p.bg[0], C0);
    p.out_rgb[3 * (size_t)ray + 1] = fmaf(bgw, p.bg[1], C1);
    p.out_rgb[3 * (size_t)ray + 2] = fmaf(bgw, p.bg[2], C2);
    if (DBG) {
        if (p.flags & FPO_FLAG_OUT_T) p.out_T[ray] = T;
        if (p.flags & FPO_FLAG_RECORD_VISITS) p.visit_count[ray] = n_visits;
    }
}

}  // namespace

// Persistent kernel: a grid of (SM count x resident CTAs) pulls warp-sized
// tiles (8x4 pixels, or 32 consecutive explicit rays) from one atomic
// counter.  Each CTA first stages the top n_smem_nodes nodes of the
// breadth-first node array and the frame constants in shared memory.  The
// last CTA to finish resets the counter for the next launch.
template <bool MAT, bool DBG, int N1, int N2>
__global__ void __launch_bounds__(TRAV_THREADS) traverse_kernel(const __grid_constant__ TraverseParams p)
{
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ FrameShared fs;
    uint32_t *s_nodes = smem;
    uint32_t *s_stack = smem + p.n_smem_nodes * 8;

    {
        const uint4 *src = reinterpret_cast<const uint4 *>(p.nodes);
        uint4 *dst = reinterpret_cast<uint4 *>(s_nodes);
        for (uint32_t i = threadIdx.x; i < p.n_smem_nodes * 2; i += blockDim.x) dst[i] = __ldg(src + i);
        const int nb = p.n1 > p.n2 ? p.n1 : p.n2;
        if (threadIdx.x < MAX_BASIS)
            fs.b[threadIdx.x] = (int)threadIdx.x < nb ? basis_fp64(threadIdx.x, p.fr.t, p.fr.period_T) : 0.0f;
        if (threadIdx.x == MAX_BASIS && p.fr.mode == FPO_RAYS_CAMERA) {
            double f[3], r[3], u[3];
            for (int k = 0; k < 3; ++k) f[k] = p.fr.target[k] - p.fr.eye[k];
            double fl = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
            for (int k = 0; k < 3; ++k) f[k] /= fl;
            r[0] = f[1] * p.fr.up[2] - f[2] * p.fr.up[1];
            r[1] = f[2] * p.fr.up[0] - f[0] * p.fr.up[2];
            r[2] = f[0] * p.fr.up[1] - f[1] * p.fr.up[0];
            double rl = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
            for (int k = 0; k < 3; ++k) r[k] /= rl;
            u[0] = r[1] * f[2] - r[2] * f[1];
            u[1] = r[2] * f[0] - r[0] * f[2];
            u[2] = r[0] * f[1] - r[1] * f[0];
            const double th = tan(0.5 * p.fr.fov_y_deg * 3.14159265358979323846 / 180.0);
            for (int k = 0; k < 3; ++k) {
                fs.f[k] = (float)f[k];
                fs.r[k] = (float)r[k];
                fs.u[k] = (float)u[k];
                fs.eye[k] = (float)p.fr.eye[k];
            }
            fs.sx_scale = (float)(th * (double)p.fr.width / (double)p.fr.height);
            fs.sy_scale = (float)th;
        }
    }
    __syncthreads();

    const int lane = threadIdx.x & 31;
    uint32_t *my_stack = s_stack + threadIdx.x;
    for (;;) {
        uint32_t tile = 0;
        if (lane == 0) tile = atomicAdd(p.status + 1, 1u);
        tile = __shfl_sync(0xffffffffu, tile, 0);
        if (tile >= p.n_tiles) break;
        uint32_t ray;
        int px = 0, py = 0;
        bool valid;
        if (p.fr.mode == FPO_RAYS_CAMERA) {
            const uint32_t tx = tile % p.tiles_x, ty = tile / p.tiles_x;
            px = (int)(tx * 8 + (lane & 7));
            py = (int)(ty * 4 + (lane >> 3));
            valid = px < (int)p.fr.width && py < (int)p.fr.height;
            ray = (uint32_t)py * p.fr.width + (uint32_t)px;
        } else {
            ray = tile * 32 + lane;
            valid = ray < p.fr.n_rays;
        }
        if (valid) trace_ray<MAT, DBG, N1, N2>(p, fs, s_nodes, my_stack, TRAV_THREADS, ray, px, py);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t done = atomicAdd(p.status + 2, 1u);
        if (done == gridDim.x - 1) {
            atomicExch(p.status + 1, 0u);
            atomicExch(p.status + 2, 0u);
        }
    }
}

int traverse_smem_bytes(uint32_t n_smem_nodes)
{
    return (int)(n_smem_nodes * 32u + STACK_LEVELS * TRAV_THREADS * 4u);
}

int traverse_block_threads() { return TRAV_THREADS; }

template <bool MAT, bool DBG, int N1, int N2>
static int launch_t(const TraverseParams &p, int sm_count, cudaStream_t s)
{
    const int smem = traverse_smem_bytes(p.n_smem_nodes);
    auto k = traverse_kernel<MAT, DBG, N1, N2>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return (int)e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, TRAV_THREADS, smem);
    if (e != cudaSuccess) return (int)e;
    if (per_sm < 1) per_sm = 1;
    uint64_t blocks = (uint64_t)sm_count * per_sm;
    const uint64_t need = (p.n_tiles + (TRAV_THREADS / 32) - 1) / (TRAV_THREADS / 32);
    if (need < blocks) blocks = need ? need : 1;
    k<<<(unsigned)blocks, TRAV_THREADS, smem, s>>>(p);
    return (int)cudaGetLastError();
}

template <bool DBG>
static int launch_fused(const TraverseParams &p, int sm_count, cudaStream_t s)
{
    // Fused per-visit IDFT: compile-time Fourier sizes (the settings of Tab. 3).
    if (p.n1 == 31 && p.n2 == 5) return launch_t<false, DBG, 31, 5>(p, sm_count, s);
    if (p.n1 == 11 && p.n2 == 5) return launch_t<false, DBG, 11, 5>(p, sm_count, s);
    if (p.n1 == 21 && p.n2 == 5) return launch_t<false, DBG, 21, 5>(p, sm_count, s);
    if (p.n1 == 31 && p.n2 == 11) return launch_t<false, DBG, 31, 11>(p, sm_count, s);
    return -1;
}

bool fused_supported(int n1, int n2)
{
    return (n1 == 31 && n2 == 5) || (n1 == 11 && n2 == 5) || (n1 == 21 && n2 == 5) ||
           (n1 == 31 && n2 == 11);
}

int launch_traverse(const TraverseParams &p, bool materialised, bool debug, int sm_count,
                    void *stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    if (materialised)
        return debug ? launch_t<true, true, 0, 0>(p, sm_count, s) : launch_t<true, false, 0, 0>(p, sm_count, s);
    return debug ? launch_fused<true>(p, sm_count, s) : launch_fused<false>(p, sm_count, s);
}

}  // namespace fpo
