// Training kernels of the latent decoder (FP32 masters, SIMT):
//
//  decoder_grad_kernel  for a batch of leaves, the MLP forward
//                       (32 -> 64 -> 64 -> n1 + 27 n2, ReLU), the weighted L2
//                       loss against target coefficients (plus an optional
//                       extra dL/dy, e.g. from the render adjoint), and the
//                       back-propagation to the latents and to every weight.
//                       Each CTA keeps all weights in shared memory, walks
//                       tiles of 64 leaves with register-tiled products, sums
//                       its weight gradients in registers, and adds them to
//                       the global gradients once at the end.
//  adam_kernel          Adam (Kingma & Ba) on a dense array or on the rows of
//                       a batch (distinct rows).
//  leaf_adam_kernel     Adam on the marked leaves' coefficient rows, written
//                       back into the renderer's FP32 records.
#include <cuda_runtime.h>

#include <cstdint>

#include "fpo_internal.h"

namespace fpo {
namespace {

// Tiles of TG_ROWS leaves; thread (tr, tc) = (tid >> 4, tid & 15) owns rows
// 4 tr .. 4 tr + 3 and the outputs tc + 16 j of each activation layer, and the
// weight-gradient entries (tc + 16 j, tr + 16 i) of each layer, summed in
// registers over all of its CTA's tiles.  Weights are kept as [out][in] rows
// padded to in + 1 floats, activations as [row][feature] rows padded the same
// way: a warp then reads 16 consecutive words or a broadcast whichever index
// it varies, so no shared-memory read has a bank conflict.
constexpr int TG_THREADS = 256;
constexpr int TG_ROWS = 64;   // leaves per tile
constexpr int TG_MAXC = 176;  // n1 + 27 n2 <= 176 (31 + 135 = 166)
constexpr int TG_J = TG_MAXC / 16;
constexpr int S1 = 33, S2 = 65, SY = TG_MAXC + 1;  // padded row strides

struct GradSmem {
    float w1[64 * S1], w2[64 * S2], w3[TG_MAXC * S2], b1[64], b2[64], b3[TG_MAXC];
    float x[TG_ROWS * S1], h1[TG_ROWS * S2], h2[TG_ROWS * S2], dy[TG_ROWS * SY];
    float d2[TG_ROWS * S2], d1[TG_ROWS * S2];
    uint32_t row[TG_ROWS];
    double loss;
};

}  // namespace

__global__ void __launch_bounds__(TG_THREADS, 1) decoder_grad_kernel(const __grid_constant__ DecoderGradParams p)
{
    extern __shared__ __align__(16) unsigned char tg_raw[];
    GradSmem &S = *reinterpret_cast<GradSmem *>(tg_raw);
    const int tid = threadIdx.x, nc = p.nc;
    const int tr = tid >> 4, tc = tid & 15;
    for (int i = tid; i < 64 * 32; i += TG_THREADS) S.w1[(i >> 5) * S1 + (i & 31)] = p.w.w1[i];
    for (int i = tid; i < 64 * 64; i += TG_THREADS) S.w2[(i >> 6) * S2 + (i & 63)] = p.w.w2[i];
    for (int i = tid; i < TG_MAXC * 64; i += TG_THREADS) {
        const int j = i >> 6;
        S.w3[j * S2 + (i & 63)] = j < nc ? p.w.w3[i] : 0.0f;
    }
    for (int i = tid; i < 64; i += TG_THREADS) { S.b1[i] = p.w.b1[i]; S.b2[i] = p.w.b2[i]; }
    for (int i = tid; i < TG_MAXC; i += TG_THREADS) S.b3[i] = i < nc ? p.w.b3[i] : 0.0f;
    if (tid == 0) S.loss = 0.0;

    float g3[TG_J][4], g2[4][4], g1[4][2], gb = 0.0f, gb2 = 0.0f, gb1 = 0.0f, lsum = 0.0f;
#pragma unroll
    for (int j = 0; j < TG_J; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) g3[j][i] = 0.0f;
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) g2[j][i] = 0.0f;
#pragma unroll
    for (int j = 0; j < 4; ++j) g1[j][0] = g1[j][1] = 0.0f;

    const uint32_t n_tiles = (p.batch + TG_ROWS - 1) / TG_ROWS;
    for (uint32_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const uint32_t r0 = tile * TG_ROWS;
        const int nr = (int)min((uint32_t)TG_ROWS, p.batch - r0);
        __syncthreads();  // weights staged; the previous tile is done with every buffer
        if (tid < TG_ROWS) S.row[tid] = tid < nr ? p.rows[r0 + tid] : 0u;
        __syncthreads();
        for (int i = tid; i < TG_ROWS * 32; i += TG_THREADS) {
            const int r = i >> 5;
            S.x[r * S1 + (i & 31)] = r < nr ? p.latents[(size_t)S.row[r] * 32 + (i & 31)] : 0.0f;
        }
        __syncthreads();
        // h1 = relu(W1 x + b1)
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
                for (int i = 0; i < 4; ++i) xv[i] = S.x[(4 * tr + i) * S1 + k];
#pragma unroll
                for (int j = 0; j < 4; ++j) wv[j] = S.w1[(tc + 16 * j) * S1 + k];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) a[i][j] = fmaf(xv[i], wv[j], a[i][j]);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) S.h1[(4 * tr + i) * S2 + tc + 16 * j] = fmaxf(a[i][j], 0.0f);
        }
        __syncthreads();
        // h2 = relu(W2 h1 + b2)
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
                for (int i = 0; i < 4; ++i) xv[i] = S.h1[(4 * tr + i) * S2 + k];
#pragma unroll
                for (int j = 0; j < 4; ++j) wv[j] = S.w2[(tc + 16 * j) * S2 + k];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) a[i][j] = fmaf(xv[i], wv[j], a[i][j]);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) S.h2[(4 * tr + i) * S2 + tc + 16 * j] = fmaxf(a[i][j], 0.0f);
        }
        __syncthreads();
        // y = W3 h2 + b3; dy = 2 cw (y - target) + extra (0 on padding rows and columns)
        {
            float a[4][TG_J];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < TG_J; ++j) a[i][j] = S.b3[tc + 16 * j];
#pragma unroll 2
            for (int k = 0; k < 64; ++k) {
                float xv[4], wv[TG_J];
#pragma unroll
                for (int i = 0; i < 4; ++i) xv[i] = S.h2[(4 * tr + i) * S2 + k];
#pragma unroll
                for (int j = 0; j < TG_J; ++j) wv[j] = S.w3[(tc + 16 * j) * S2 + k];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < TG_J; ++j) a[i][j] = fmaf(xv[i], wv[j], a[i][j]);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int r = 4 * tr + i;
                const size_t row = S.row[r];
#pragma unroll
                for (int j = 0; j < TG_J; ++j) {
                    const int c = tc + 16 * j;
                    float d = 0.0f;
                    if (r < nr && c < nc) {
                        const float e = a[i][j] - p.targets[row * nc + c];
                        const float cw = p.coef_weight[c];
                        lsum = fmaf(cw * e, e, lsum);
                        d = 2.0f * cw * e;
                        if (p.extra_dy) d += p.extra_dy[row * nc + c];
                    }
                    S.dy[r * SY + c] = d;
                }
            }
        }
        __syncthreads();
        // d2 = (W3^T dy) * [h2 > 0];  g3 += dy h2^T;  gb3 += dy
        {
            float a[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) a[i][j] = 0.0f;
#pragma unroll 2
            for (int c = 0; c < nc; ++c) {
                float dv[4], wv[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) dv[i] = S.dy[(4 * tr + i) * SY + c];
#pragma unroll
                for (int j = 0; j < 4; ++j) wv[j] = S.w3[c * S2 + tc + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) a[i][j] = fmaf(dv[i], wv[j], a[i][j]);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int o = (4 * tr + i) * S2 + tc + 16 * j;
                    S.d2[o] = S.h2[o] > 0.0f ? a[i][j] : 0.0f;
                }
#pragma unroll 2
            for (int r = 0; r < nr; ++r) {
                float dv[TG_J], hv[4];
#pragma unroll
                for (int j = 0; j < TG_J; ++j) dv[j] = S.dy[r * SY + tc + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; ++i) hv[i] = S.h2[r * S2 + tr + 16 * i];
#pragma unroll
                for (int j = 0; j < TG_J; ++j)
#pragma unroll
                    for (int i = 0; i < 4; ++i) g3[j][i] = fmaf(dv[j], hv[i], g3[j][i]);
            }
            if (tid < nc)
                for (int r = 0; r < nr; ++r) gb += S.dy[r * SY + tid];
        }
        __syncthreads();
        // d1 = (W2^T d2) * [h1 > 0];  g2 += d2 h1^T;  gb2 += d2
        {
            float a[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) a[i][j] = 0.0f;
#pragma unroll 4
            for (int o = 0; o < 64; ++o) {
                float dv[4], wv[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) dv[i] = S.d2[(4 * tr + i) * S2 + o];
#pragma unroll
                for (int j = 0; j < 4; ++j) wv[j] = S.w2[o * S2 + tc + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) a[i][j] = fmaf(dv[i], wv[j], a[i][j]);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int o = (4 * tr + i) * S2 + tc + 16 * j;
                    S.d1[o] = S.h1[o] > 0.0f ? a[i][j] : 0.0f;
                }
#pragma unroll 4
            for (int r = 0; r < nr; ++r) {
                float dv[4], hv[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) dv[j] = S.d2[r * S2 + tc + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; ++i) hv[i] = S.h1[r * S2 + tr + 16 * i];
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int i = 0; i < 4; ++i) g2[j][i] = fmaf(dv[j], hv[i], g2[j][i]);
            }
            if (tid < 64)
                for (int r = 0; r < nr; ++r) gb2 += S.d2[r * S2 + tid];
        }
        __syncthreads();
        // dx = W1^T d1 (the latents' gradient);  g1 += d1 x^T;  gb1 += d1
        {
            float a[4][2];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i][0] = a[i][1] = 0.0f;
#pragma unroll 4
            for (int o = 0; o < 64; ++o) {
                float dv[4], wv[2];
#pragma unroll
                for (int i = 0; i < 4; ++i) dv[i] = S.d1[(4 * tr + i) * S2 + o];
#pragma unroll
                for (int j = 0; j < 2; ++j) wv[j] = S.w1[o * S1 + tc + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 2; ++j) a[i][j] = fmaf(dv[i], wv[j], a[i][j]);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int r = 4 * tr + i;
                if (r < nr) {
                    p.dlatents[(size_t)(r0 + r) * 32 + tc] = a[i][0];
                    p.dlatents[(size_t)(r0 + r) * 32 + tc + 16] = a[i][1];
                }
            }
#pragma unroll 4
            for (int r = 0; r < nr; ++r) {
                float dv[4], xv[2];
#pragma unroll
                for (int j = 0; j < 4; ++j) dv[j] = S.d1[r * S2 + tc + 16 * j];
#pragma unroll
                for (int i = 0; i < 2; ++i) xv[i] = S.x[r * S1 + tr + 16 * i];
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int i = 0; i < 2; ++i) g1[j][i] = fmaf(dv[j], xv[i], g1[j][i]);
            }
            if (tid < 64)
                for (int r = 0; r < nr; ++r) gb1 += S.d1[r * S2 + tid];
        }
    }
    // this CTA's sums into the global gradients
#pragma unroll
    for (int j = 0; j < TG_J; ++j)
        if (tc + 16 * j < nc) {
#pragma unroll
            for (int i = 0; i < 4; ++i) atomicAdd(p.g.w3 + (tc + 16 * j) * 64 + tr + 16 * i, g3[j][i]);
        }
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) atomicAdd(p.g.w2 + (tc + 16 * j) * 64 + tr + 16 * i, g2[j][i]);
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 2; ++i) atomicAdd(p.g.w1 + (tc + 16 * j) * 32 + tr + 16 * i, g1[j][i]);
    if (tid < nc) atomicAdd(p.g.b3 + tid, gb);
    if (tid < 64) {
        atomicAdd(p.g.b2 + tid, gb2);
        atomicAdd(p.g.b1 + tid, gb1);
    }
    // loss: warp sums, then one shared double per CTA
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    __syncthreads();
    if ((tid & 31) == 0) atomicAdd(&S.loss, (double)lsum);
    __syncthreads();
    if (tid == 0 && p.loss) atomicAdd(p.loss, S.loss);
}

int launch_decoder_grad(const DecoderGradParams &p, int sm_count, void *stream)
{
    if (p.batch == 0) return (int)cudaSuccess;
    const int smem = (int)sizeof(GradSmem);
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
// each thread owns 4 rows x the output columns 4 tc + 64 g + e (e = 0..3; g = 0
// for the 64-wide hidden layers, g = 0..2 for the last layer), so per input
// feature it reads its weights with one 16-byte load per group (16 threads
// read 256 consecutive bytes) and its 4 activations as broadcasts.  In the
// last layer, columns 176..191 of group 2 read into the next weight row (or the
// biases after it) and are discarded.
// Record mode (perm != nullptr): output row i is the context's FP32 record
// i, decoded from latent row perm[i], its first n1 values going to the
// density records (stride ss) and the rest to the SH records (stride zs).
constexpr int DF_ROWS = 64, DF_THREADS = 256, DF_MAXC = 176;

struct DecodeSmem {
    float w1t[32 * 64], w2t[64 * 64], w3t[64 * DF_MAXC], b1[64], b2[64], b3[DF_MAXC + 16];
    float x[DF_ROWS * 33], h1[DF_ROWS * 65], h2[DF_ROWS * 65];
    uint32_t src[DF_ROWS];
};

struct DecodeOut {
    float *coeffs;          // [n][nc], or nullptr in record mode
    const uint32_t *perm;   // record -> latent row (record mode)
    float *sig, *zc;        // FP32 records (record mode)
    int n1, ss, zs;
};

// a[i][4 g + e] += sum_k in[(4 tr + i) * ld_in + k] * wt[k * ldw + 4 tc + 64 g + e]
template <int G>
__device__ __forceinline__ void decode_layer(const float *in, int ld_in, int K, const float *wt, int ldw,
                                             float (&a)[4][4 * G], int tr, int tc)
{
#pragma unroll 2
    for (int k = 0; k < K; ++k) {
        float xv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) xv[i] = in[(4 * tr + i) * ld_in + k];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const float4 w = *reinterpret_cast<const float4 *>(wt + k * ldw + 4 * tc + 64 * g);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                a[i][4 * g] = fmaf(xv[i], w.x, a[i][4 * g]);
                a[i][4 * g + 1] = fmaf(xv[i], w.y, a[i][4 * g + 1]);
                a[i][4 * g + 2] = fmaf(xv[i], w.z, a[i][4 * g + 2]);
                a[i][4 * g + 3] = fmaf(xv[i], w.w, a[i][4 * g + 3]);
            }
        }
    }
}

__global__ void __launch_bounds__(DF_THREADS, 2) decoder_forward_kernel(const fpo_mlp w, int nc, uint32_t n,
                                                                         const float *__restrict__ latents,
                                                                         const DecodeOut o)
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
    for (int i = tid; i < DF_MAXC + 16; i += DF_THREADS) S.b3[i] = i < nc ? w.b3[i] : 0.0f;
    const int tr = tid >> 4, tc = tid & 15;  // rows 4 tr .. 4 tr + 3; columns 4 tc + 64 g + e
    const uint32_t n_tiles = (n + DF_ROWS - 1) / DF_ROWS;
    for (uint32_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const uint32_t r0 = tile * DF_ROWS;
        const int nr = (int)min((uint32_t)DF_ROWS, n - r0);
        __syncthreads();  // weights staged; the previous tile is done with x, h1, h2, src
        if (tid < DF_ROWS) S.src[tid] = tid < nr ? (o.perm ? o.perm[r0 + tid] : r0 + tid) : 0u;
        __syncthreads();
        for (int i = tid; i < DF_ROWS * 32; i += DF_THREADS) {
            const int r = i >> 5;
            S.x[r * 33 + (i & 31)] = r < nr ? latents[(size_t)S.src[r] * 32 + (i & 31)] : 0.0f;
        }
        __syncthreads();
        {
            float a[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int e = 0; e < 4; ++e) a[i][e] = S.b1[4 * tc + e];
            decode_layer<1>(S.x, 33, 32, S.w1t, 64, a, tr, tc);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int e = 0; e < 4; ++e) S.h1[(4 * tr + i) * 65 + 4 * tc + e] = fmaxf(a[i][e], 0.0f);
        }
        __syncthreads();
        {
            float a[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int e = 0; e < 4; ++e) a[i][e] = S.b2[4 * tc + e];
            decode_layer<1>(S.h1, 65, 64, S.w2t, 64, a, tr, tc);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int e = 0; e < 4; ++e) S.h2[(4 * tr + i) * 65 + 4 * tc + e] = fmaxf(a[i][e], 0.0f);
        }
        __syncthreads();
        {
            float a[4][12];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 12; ++j) a[i][j] = S.b3[4 * tc + 64 * (j >> 2) + (j & 3)];
            decode_layer<3>(S.h2, 65, 64, S.w3t, DF_MAXC, a, tr, tc);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int r = 4 * tr + i;
                if (r < nr) {
                    const size_t row = r0 + r;
#pragma unroll
                    for (int j = 0; j < 12; ++j) {
                        const int c = 4 * tc + 64 * (j >> 2) + (j & 3);
                        if (c >= nc) continue;
                        if (!o.perm) o.coeffs[row * nc + c] = a[i][j];
                        else if (c < o.n1) o.sig[row * o.ss + c] = a[i][j];
                        else o.zc[row * o.zs + (c - o.n1)] = a[i][j];
                    }
                }
            }
        }
    }
}

static int launch_decode(const fpo_mlp &w, int nc, uint32_t n, const float *latents, const DecodeOut &o,
                         int sm_count, void *stream)
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
    decoder_forward_kernel<<<(unsigned)blocks, DF_THREADS, smem, (cudaStream_t)stream>>>(w, nc, n, latents, o);
    return (int)cudaGetLastError();
}

int launch_decoder_forward(const fpo_mlp &w, int nc, uint32_t n, const float *latents, float *out, int sm_count,
                           void *stream)
{
    DecodeOut o{};
    o.coeffs = out;
    return launch_decode(w, nc, n, latents, o, sm_count, stream);
}

int launch_decode_records(const fpo_mlp &w, int n1, int n2, uint32_t n, const float *latents, const uint32_t *perm,
                          float *sig, float *zc, int sm_count, void *stream)
{
    DecodeOut o{};
    o.perm = perm;
    o.sig = sig;
    o.zc = zc;
    o.n1 = n1;
    o.ss = sig_stride(n1);
    o.zs = z_stride(n2);
    return launch_decode(w, n1 + 27 * n2, n, latents, o, sm_count, stream);
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
