// Training kernels of the latent decoder (FP32 masters, SIMT):
//
//  decoder_grad_kernel  for a batch of leaves, the MLP forward
//                       (32 -> 64 -> 64 -> n1 + 27 n2, ReLU), the weighted L2
//                       loss against target coefficients (plus an optional
//                       extra dL/dy, e.g. from the render adjoint), and the
//                       back-propagation to the latents and to every weight.
//                       Each CTA keeps all weights and its own weight-gradient
//                       sums in shared memory, walks tiles of 32 leaves, and
//                       adds its sums to the global gradients once at the end.
//  adam_kernel          Adam (Kingma & Ba) on a dense array or on the rows of
//                       a batch (distinct rows).
//  leaf_adam_kernel     Adam on the marked leaves' coefficient rows, written
//                       back into the renderer's FP32 records.
#include <cuda_runtime.h>

#include <cstdint>

#include "fpo_internal.h"

namespace fpo {
namespace {

constexpr int TG_THREADS = 256;
constexpr int TG_ROWS = 32;   // leaves per tile
constexpr int TG_MAXC = 176;  // n1 + 27 n2 <= 176 (31 + 135 = 166)

struct Smem {
    float w1[64 * 32], b1[64], w2[64 * 64], b2[64], w3[TG_MAXC * 64], b3[TG_MAXC];
    float g1[64 * 32], gb1[64], g2[64 * 64], gb2[64], g3[TG_MAXC * 64], gb3[TG_MAXC];
    float x[TG_ROWS * 32], z1[TG_ROWS * 64], z2[TG_ROWS * 64], dy[TG_ROWS * TG_MAXC];
    float d2[TG_ROWS * 64], d1[TG_ROWS * 64];
    double loss;
};

}  // namespace

__global__ void __launch_bounds__(TG_THREADS) decoder_grad_kernel(const __grid_constant__ DecoderGradParams p)
{
    extern __shared__ __align__(16) unsigned char tg_raw[];
    Smem &S = *reinterpret_cast<Smem *>(tg_raw);
    const int tid = threadIdx.x, nc = p.nc;
    for (int i = tid; i < 64 * 32; i += TG_THREADS) { S.w1[i] = p.w.w1[i]; S.g1[i] = 0.0f; }
    for (int i = tid; i < 64 * 64; i += TG_THREADS) { S.w2[i] = p.w.w2[i]; S.g2[i] = 0.0f; }
    for (int i = tid; i < nc * 64; i += TG_THREADS) { S.w3[i] = p.w.w3[i]; S.g3[i] = 0.0f; }
    for (int i = tid; i < 64; i += TG_THREADS) { S.b1[i] = p.w.b1[i]; S.b2[i] = p.w.b2[i]; S.gb1[i] = 0.0f; S.gb2[i] = 0.0f; }
    for (int i = tid; i < nc; i += TG_THREADS) { S.b3[i] = p.w.b3[i]; S.gb3[i] = 0.0f; }
    if (tid == 0) S.loss = 0.0;
    __syncthreads();
    const uint32_t n_tiles = (p.batch + TG_ROWS - 1) / TG_ROWS;
    for (uint32_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const uint32_t r0 = tile * TG_ROWS;
        const int nr = (int)min((uint32_t)TG_ROWS, p.batch - r0);
        for (int i = tid; i < TG_ROWS * 32; i += TG_THREADS) {
            const int r = i >> 5;
            S.x[i] = r < nr ? p.latents[(size_t)p.rows[r0 + r] * 32 + (i & 31)] : 0.0f;
        }
        __syncthreads();
        // z1 = W1 x + b1
        for (int i = tid; i < TG_ROWS * 64; i += TG_THREADS) {
            const int r = i >> 6, o = i & 63;
            float a = S.b1[o];
#pragma unroll 8
            for (int k = 0; k < 32; ++k) a = fmaf(S.w1[o * 32 + k], S.x[r * 32 + k], a);
            S.z1[i] = a;
        }
        __syncthreads();
        // z2 = W2 relu(z1) + b2
        for (int i = tid; i < TG_ROWS * 64; i += TG_THREADS) {
            const int r = i >> 6, o = i & 63;
            float a = S.b2[o];
#pragma unroll 8
            for (int k = 0; k < 64; ++k) a = fmaf(S.w2[o * 64 + k], fmaxf(S.z1[r * 64 + k], 0.0f), a);
            S.z2[i] = a;
        }
        __syncthreads();
        // y = W3 relu(z2) + b3; dy = 2 cw (y - target) + extra
        float lsum = 0.0f;
        for (int i = tid; i < TG_ROWS * nc; i += TG_THREADS) {
            const int r = i / nc, j = i % nc;
            float d = 0.0f;
            if (r < nr) {
                float a = S.b3[j];
#pragma unroll 8
                for (int k = 0; k < 64; ++k) a = fmaf(S.w3[j * 64 + k], fmaxf(S.z2[r * 64 + k], 0.0f), a);
                const size_t row = p.rows[r0 + r];
                const float e = a - p.targets[row * nc + j];
                const float cw = p.coef_weight[j];
                lsum += cw * e * e;
                d = 2.0f * cw * e;
                if (p.extra_dy) d += p.extra_dy[row * nc + j];
            }
            S.dy[r * TG_MAXC + j] = d;
        }
        atomicAdd(&S.loss, (double)lsum);
        __syncthreads();
        // d2 = (W3^T dy) * [z2 > 0]; g3 += dy relu(z2)^T; gb3 += dy
        for (int i = tid; i < TG_ROWS * 64; i += TG_THREADS) {
            const int r = i >> 6, k = i & 63;
            float a = 0.0f;
            for (int j = 0; j < nc; ++j) a = fmaf(S.dy[r * TG_MAXC + j], S.w3[j * 64 + k], a);
            S.d2[i] = S.z2[i] > 0.0f ? a : 0.0f;
        }
        for (int i = tid; i < nc * 64; i += TG_THREADS) {
            const int j = i >> 6, k = i & 63;
            float a = 0.0f;
            for (int r = 0; r < nr; ++r) a = fmaf(S.dy[r * TG_MAXC + j], fmaxf(S.z2[r * 64 + k], 0.0f), a);
            S.g3[i] += a;
        }
        for (int j = tid; j < nc; j += TG_THREADS) {
            float a = 0.0f;
            for (int r = 0; r < nr; ++r) a += S.dy[r * TG_MAXC + j];
            S.gb3[j] += a;
        }
        __syncthreads();
        // d1 = (W2^T d2) * [z1 > 0]; g2 += d2 relu(z1)^T; gb2 += d2
        for (int i = tid; i < TG_ROWS * 64; i += TG_THREADS) {
            const int r = i >> 6, k = i & 63;
            float a = 0.0f;
#pragma unroll 8
            for (int o = 0; o < 64; ++o) a = fmaf(S.d2[r * 64 + o], S.w2[o * 64 + k], a);
            S.d1[i] = S.z1[i] > 0.0f ? a : 0.0f;
        }
        for (int i = tid; i < 64 * 64; i += TG_THREADS) {
            const int o = i >> 6, k = i & 63;
            float a = 0.0f;
            for (int r = 0; r < nr; ++r) a = fmaf(S.d2[r * 64 + o], fmaxf(S.z1[r * 64 + k], 0.0f), a);
            S.g2[i] += a;
        }
        for (int o = tid; o < 64; o += TG_THREADS) {
            float a = 0.0f;
            for (int r = 0; r < nr; ++r) a += S.d2[r * 64 + o];
            S.gb2[o] += a;
        }
        __syncthreads();
        // dx = W1^T d1; g1 += d1 x^T; gb1 += d1
        for (int i = tid; i < TG_ROWS * 32; i += TG_THREADS) {
            const int r = i >> 5, k = i & 31;
            if (r < nr) {
                float a = 0.0f;
#pragma unroll 8
                for (int o = 0; o < 64; ++o) a = fmaf(S.d1[r * 64 + o], S.w1[o * 32 + k], a);
                p.dlatents[(size_t)(r0 + r) * 32 + k] = a;
            }
        }
        for (int i = tid; i < 64 * 32; i += TG_THREADS) {
            const int o = i >> 5, k = i & 31;
            float a = 0.0f;
            for (int r = 0; r < nr; ++r) a = fmaf(S.d1[r * 64 + o], S.x[r * 32 + k], a);
            S.g1[i] += a;
        }
        for (int o = tid; o < 64; o += TG_THREADS) {
            float a = 0.0f;
            for (int r = 0; r < nr; ++r) a += S.d1[r * 64 + o];
            S.gb1[o] += a;
        }
        __syncthreads();
    }
    for (int i = tid; i < 64 * 32; i += TG_THREADS) atomicAdd(p.g.w1 + i, S.g1[i]);
    for (int i = tid; i < 64 * 64; i += TG_THREADS) atomicAdd(p.g.w2 + i, S.g2[i]);
    for (int i = tid; i < nc * 64; i += TG_THREADS) atomicAdd(p.g.w3 + i, S.g3[i]);
    for (int i = tid; i < 64; i += TG_THREADS) { atomicAdd(p.g.b1 + i, S.gb1[i]); atomicAdd(p.g.b2 + i, S.gb2[i]); }
    for (int i = tid; i < nc; i += TG_THREADS) atomicAdd(p.g.b3 + i, S.gb3[i]);
    if (tid == 0 && p.loss) atomicAdd(p.loss, S.loss);
}

int launch_decoder_grad(const DecoderGradParams &p, int sm_count, void *stream)
{
    if (p.batch == 0) return (int)cudaSuccess;
    const int smem = (int)sizeof(Smem);
    cudaError_t e = cudaFuncSetAttribute(decoder_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return (int)e;
    const uint32_t n_tiles = (p.batch + TG_ROWS - 1) / TG_ROWS;
    uint32_t blocks = (uint32_t)sm_count;
    if (blocks > n_tiles) blocks = n_tiles;
    decoder_grad_kernel<<<blocks, TG_THREADS, smem, (cudaStream_t)stream>>>(p);
    return (int)cudaGetLastError();
}

int decoder_grad_max_coeffs() { return TG_MAXC; }

// FP32 decode of every leaf: y = W3 relu(W2 relu(W1 x + b1) + b2) + b3.  A CTA
// keeps the transposed weights in shared memory and walks tiles of 64 leaves;
// each thread owns 4 rows x (outputs tc, tc + 16, ...) of a layer, so a warp
// reads weight rows without bank conflicts and activations as broadcasts.
constexpr int DF_ROWS = 64, DF_THREADS = 256, DF_MAXC = 176;

struct DecodeSmem {
    float w1t[32 * 64], w2t[64 * 64], w3t[64 * DF_MAXC], b1[64], b2[64], b3[DF_MAXC];
    float x[DF_ROWS * 33], h1[DF_ROWS * 65], h2[DF_ROWS * 65];
};

__global__ void __launch_bounds__(DF_THREADS) decoder_forward_kernel(const fpo_mlp w, int nc, uint32_t n,
                                                                      const float *__restrict__ latents,
                                                                      float *__restrict__ out)
{
    extern __shared__ __align__(16) unsigned char df_raw[];
    DecodeSmem &S = *reinterpret_cast<DecodeSmem *>(df_raw);
    const int tid = threadIdx.x;
    for (int i = tid; i < 64 * 32; i += DF_THREADS) S.w1t[(i & 31) * 64 + (i >> 5)] = w.w1[i];
    for (int i = tid; i < 64 * 64; i += DF_THREADS) S.w2t[(i & 63) * 64 + (i >> 6)] = w.w2[i];
    for (int i = tid; i < DF_MAXC * 64; i += DF_THREADS) {
        const int c = i >> 6, k = i & 63;
        S.w3t[k * DF_MAXC + c] = c < nc ? w.w3[c * 64 + k] : 0.0f;
    }
    for (int i = tid; i < 64; i += DF_THREADS) { S.b1[i] = w.b1[i]; S.b2[i] = w.b2[i]; }
    for (int i = tid; i < DF_MAXC; i += DF_THREADS) S.b3[i] = i < nc ? w.b3[i] : 0.0f;
    const int tr = tid >> 4, tc = tid & 15;  // rows 4 tr .. 4 tr + 3; outputs tc + 16 j
    const uint32_t n_tiles = (n + DF_ROWS - 1) / DF_ROWS;
    for (uint32_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const uint32_t r0 = tile * DF_ROWS;
        const int nr = (int)min((uint32_t)DF_ROWS, n - r0);
        __syncthreads();  // weights staged; the previous tile is done with x, h1, h2
        for (int i = tid; i < DF_ROWS * 32; i += DF_THREADS) {
            const int r = i >> 5;
            S.x[r * 33 + (i & 31)] = r < nr ? latents[(size_t)(r0 + r) * 32 + (i & 31)] : 0.0f;
        }
        __syncthreads();
        {
            float a[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) a[i][j] = S.b1[tc + 16 * j];
#pragma unroll 4
            for (int k = 0; k < 32; ++k) {
                float xv[4], wv[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) xv[i] = S.x[(4 * tr + i) * 33 + k];
#pragma unroll
                for (int j = 0; j < 4; ++j) wv[j] = S.w1t[k * 64 + tc + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) a[i][j] = fmaf(xv[i], wv[j], a[i][j]);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) S.h1[(4 * tr + i) * 65 + tc + 16 * j] = fmaxf(a[i][j], 0.0f);
        }
        __syncthreads();
        {
            float a[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) a[i][j] = S.b2[tc + 16 * j];
#pragma unroll 4
            for (int k = 0; k < 64; ++k) {
                float xv[4], wv[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) xv[i] = S.h1[(4 * tr + i) * 65 + k];
#pragma unroll
                for (int j = 0; j < 4; ++j) wv[j] = S.w2t[k * 64 + tc + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) a[i][j] = fmaf(xv[i], wv[j], a[i][j]);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) S.h2[(4 * tr + i) * 65 + tc + 16 * j] = fmaxf(a[i][j], 0.0f);
        }
        __syncthreads();
        {
            constexpr int J = DF_MAXC / 16;
            float a[4][J];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < J; ++j) a[i][j] = S.b3[tc + 16 * j];
#pragma unroll 2
            for (int k = 0; k < 64; ++k) {
                float xv[4], wv[J];
#pragma unroll
                for (int i = 0; i < 4; ++i) xv[i] = S.h2[(4 * tr + i) * 65 + k];
#pragma unroll
                for (int j = 0; j < J; ++j) wv[j] = S.w3t[k * DF_MAXC + tc + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < J; ++j) a[i][j] = fmaf(xv[i], wv[j], a[i][j]);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int r = 4 * tr + i;
                if (r < nr) {
#pragma unroll
                    for (int j = 0; j < J; ++j)
                        if (tc + 16 * j < nc) out[(size_t)(r0 + r) * nc + tc + 16 * j] = a[i][j];
                }
            }
        }
    }
}

int launch_decoder_forward(const fpo_mlp &w, int nc, uint32_t n, const float *latents, float *out, int sm_count,
                           void *stream)
{
    if (n == 0) return (int)cudaSuccess;
    const int smem = (int)sizeof(DecodeSmem);
    cudaError_t e = cudaFuncSetAttribute(decoder_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return (int)e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, decoder_forward_kernel, DF_THREADS, smem);
    if (e != cudaSuccess) return (int)e;
    if (per_sm < 1) per_sm = 1;
    const uint32_t n_tiles = (n + DF_ROWS - 1) / DF_ROWS;
    uint64_t blocks = (uint64_t)sm_count * per_sm;
    if (blocks > n_tiles) blocks = n_tiles;
    decoder_forward_kernel<<<(unsigned)blocks, DF_THREADS, smem, (cudaStream_t)stream>>>(w, nc, n, latents, out);
    return (int)cudaGetLastError();
}

// Adam: m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
// p -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).
__global__ void adam_kernel(float *param, const float *grad, float *m, float *v, uint64_t n, const uint32_t *rows,
                            uint32_t dim, float lr, float b1, float b2, float eps, float bc1, float bc2)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const size_t at = rows ? (size_t)rows[i / dim] * dim + i % dim : (size_t)i;
        const float g = grad[i];
        const float mm = b1 * m[at] + (1.0f - b1) * g;
        const float vv = b2 * v[at] + (1.0f - b2) * g * g;
        m[at] = mm;
        v[at] = vv;
        param[at] -= lr * (mm / bc1) / (sqrtf(vv / bc2) + eps);
    }
}

int launch_adam(float *param, const float *grad, float *m, float *v, uint64_t n, const uint32_t *rows, uint32_t dim,
                float lr, float b1, float b2, float eps, uint32_t step, int sm_count, void *stream)
{
    if (n == 0) return (int)cudaSuccess;
    const double bc1 = 1.0 - pow((double)b1, (double)step), bc2 = 1.0 - pow((double)b2, (double)step);
    uint64_t blocks = (n + 255) / 256;
    if (blocks > (uint64_t)sm_count * 16) blocks = (uint64_t)sm_count * 16;
    adam_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(param, grad, m, v, n, rows, dim ? dim : 1, lr, b1,
                                                                      b2, eps, (float)bc1, (float)bc2);
    return (int)cudaGetLastError();
}

// Row-sparse Adam (Kingma & Ba) for the fine-tuning of Sec. 4.3: only the
// leaves whose mark is set (those the batch visited) are updated, as in a
// sparse-gradient Adam.  A warp takes 32 internal leaves at a time: one
// coalesced read of perm and one gather of the marks decide, by ballot, which
// of them it updates.  Marked rows go LEAF_ADAM_ROWS at a time (all their
// loads in flight together), lanes across each row's elements; every row gets
// the Adam step, goes back into the FP32 records at its internal slot, and
// has its gradient row and mark cleared for the next batch.

constexpr int LEAF_ADAM_CHUNK = 96;   // row elements per unrolled pass
constexpr int LEAF_ADAM_ROWS = 2;     // marked rows processed together

__global__ void __launch_bounds__(256, 4) leaf_adam_kernel(const __grid_constant__ LeafAdamParams p)
{
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
    const int nc = p.n1 + 27 * p.n2;
    constexpr int PER = LEAF_ADAM_CHUNK / 32;
    for (uint32_t base = warp * 32; base < p.n_leaves; base += n_warps * 32) {
        const uint32_t i = base + lane;
        uint32_t id = 0;
        bool marked = false;
        if (i < p.n_leaves) {
            id = __ldg(p.perm + i);
            marked = p.leaf_mark[id] != 0;
        }
        uint32_t todo = __ballot_sync(0xffffffffu, marked);
        while (todo) {
            uint32_t leaf[LEAF_ADAM_ROWS];
            size_t at[LEAF_ADAM_ROWS];
            bool have[LEAF_ADAM_ROWS];
#pragma unroll
            for (int r = 0; r < LEAF_ADAM_ROWS; ++r) {
                have[r] = todo != 0;
                const int src = have[r] ? __ffs(todo) - 1 : 0;
                todo &= todo - 1;
                leaf[r] = base + src;
                at[r] = (size_t)__shfl_sync(0xffffffffu, id, src) * nc;
            }
            for (int j0 = 0; j0 < nc; j0 += LEAF_ADAM_CHUNK) {
                float g[LEAF_ADAM_ROWS][PER], m[LEAF_ADAM_ROWS][PER], v[LEAF_ADAM_ROWS][PER],
                    w[LEAF_ADAM_ROWS][PER];
#pragma unroll
                for (int r = 0; r < LEAF_ADAM_ROWS; ++r)
#pragma unroll
                    for (int jj = 0; jj < PER; ++jj) {
                        const int j = j0 + lane + 32 * jj;
                        if (have[r] && j < nc) {
                            g[r][jj] = p.grad[at[r] + j];
                            m[r][jj] = p.m[at[r] + j];
                            v[r][jj] = p.v[at[r] + j];
                            w[r][jj] = p.param[at[r] + j];
                        }
                    }
#pragma unroll
                for (int r = 0; r < LEAF_ADAM_ROWS; ++r)
#pragma unroll
                    for (int jj = 0; jj < PER; ++jj) {
                        const int j = j0 + lane + 32 * jj;
                        if (have[r] && j < nc) {
                            const float mm = p.beta1 * m[r][jj] + (1.0f - p.beta1) * g[r][jj];
                            const float vv = p.beta2 * v[r][jj] + (1.0f - p.beta2) * g[r][jj] * g[r][jj];
                            const float ww = w[r][jj] - p.lr * (mm / p.bc1) / (sqrtf(vv / p.bc2) + p.eps);
                            p.m[at[r] + j] = mm;
                            p.v[at[r] + j] = vv;
                            p.param[at[r] + j] = ww;
                            p.grad[at[r] + j] = 0.0f;
                            if (j < p.n1) p.sig[(size_t)leaf[r] * p.sig_stride + j] = ww;
                            else p.zc[(size_t)leaf[r] * p.z_stride + (j - p.n1)] = ww;
                        }
                    }
            }
        }
        if (marked) p.leaf_mark[id] = 0;
    }
}

int launch_leaf_adam(const LeafAdamParams &p, int sm_count, void *stream)
{
    if (p.n_leaves == 0) return (int)cudaSuccess;
    uint64_t blocks = ((uint64_t)p.n_leaves + 255) / 256;
    if (blocks > (uint64_t)sm_count * 8) blocks = (uint64_t)sm_count * 8;
    leaf_adam_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(p);
    return (int)cudaGetLastError();
}


}  // namespace fpo

using namespace fpo;

extern "C" int fpo_decoder_grad(const fpo_mlp *w, int32_t n1, int32_t n2, uint32_t batch, const uint32_t *rows,
                                const float *latents, const float *targets, const float *coef_weight,
                                const float *extra_dy, const fpo_mlp *grad, float *dlatents, double *loss,
                                void *cuda_stream)
{
    if (!w || !grad) return set_last_error(FPO_ERR_INVALID_ARG, "NULL weights");
    if (n1 < 1 || n2 < 1 || n1 + 27 * n2 > decoder_grad_max_coeffs())
        return set_last_error(FPO_ERR_INVALID_ARG, "n1 + 27 n2 must be in [28, 176]");
    if (batch == 0) return FPO_OK;
    if (!rows || !latents || !targets || !coef_weight || !dlatents)
        return set_last_error(FPO_ERR_INVALID_ARG, "NULL array");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return set_last_error(FPO_ERR_CUDA, cudaGetErrorString(e));
    DecoderGradParams p{};
    p.w = *w;
    p.g = *grad;
    p.rows = rows;
    p.batch = batch;
    p.latents = latents;
    p.targets = targets;
    p.coef_weight = coef_weight;
    p.extra_dy = extra_dy;
    p.dlatents = dlatents;
    p.loss = loss;
    p.nc = n1 + 27 * n2;
    const int ce = launch_decoder_grad(p, sms, cuda_stream);
    if (ce != cudaSuccess) return set_last_error(FPO_ERR_CUDA, cudaGetErrorString((cudaError_t)ce));
    return FPO_OK;
}

extern "C" int fpo_decoder_forward(const fpo_mlp *w, int32_t n1, int32_t n2, uint32_t n, const float *latents,
                                   float *coeffs, void *cuda_stream)
{
    if (!w || !w->w1 || !w->b1 || !w->w2 || !w->b2 || !w->w3 || !w->b3)
        return set_last_error(FPO_ERR_INVALID_ARG, "NULL weights");
    if (n1 < 1 || n2 < 1 || n1 + 27 * n2 > DF_MAXC) return set_last_error(FPO_ERR_INVALID_ARG, "n1 + 27 n2 must be in [28, 176]");
    if (n == 0) return FPO_OK;
    if (!latents || !coeffs) return set_last_error(FPO_ERR_INVALID_ARG, "NULL array");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return set_last_error(FPO_ERR_CUDA, cudaGetErrorString(e));
    const int ce = launch_decoder_forward(*w, n1 + 27 * n2, n, latents, coeffs, sms, cuda_stream);
    if (ce != cudaSuccess) return set_last_error(FPO_ERR_CUDA, cudaGetErrorString((cudaError_t)ce));
    return FPO_OK;
}

extern "C" int fpo_adam(float *param, const float *grad, float *m, float *v, uint64_t n, const uint32_t *rows,
                        uint32_t dim, float lr, float beta1, float beta2, float eps, uint32_t step, void *cuda_stream)
{
    if (n == 0) return FPO_OK;
    if (!param || !grad || !m || !v) return set_last_error(FPO_ERR_INVALID_ARG, "NULL array");
    if (rows && dim == 0) return set_last_error(FPO_ERR_INVALID_ARG, "dim must be > 0 with rows");
    if (step < 1) return set_last_error(FPO_ERR_INVALID_ARG, "step counts from 1");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return set_last_error(FPO_ERR_CUDA, cudaGetErrorString(e));
    const int ce = launch_adam(param, grad, m, v, n, rows, dim, lr, beta1, beta2, eps, step, sms, cuda_stream);
    if (ce != cudaSuccess) return set_last_error(FPO_ERR_CUDA, cudaGetErrorString((cudaError_t)ce));
    return FPO_OK;
}
