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
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>

#include "fpo_internal.h"
#include "fpo_ptx.cuh"

#ifndef FPO_FAST_STEP
#define FPO_FAST_STEP 1
#endif
#ifndef FPO_GENERIC_NODE_LOAD
#define FPO_GENERIC_NODE_LOAD 1
#endif
// Node slots come from global memory (read-only path); 1 keeps the top
// nodes in shared memory, read through one generic pointer (measured: no gain
// alone, 1.4% slower per pipelined frame, where the 16 KB per CTA is L1).
#ifndef FPO_NODE_SMEM
#define FPO_NODE_SMEM 0
#endif
#ifndef FPO_FAST_SIGMOID
#define FPO_FAST_SIGMOID 1
#endif
#ifndef FPO_LDG256
#define FPO_LDG256 1
#endif
#ifndef FPO_PREFETCH
#define FPO_PREFETCH 1
#endif
#ifndef FPO_MAT_HALF_WARP
// FP32 records, n2 = 5, FP32 table: half (1) or a quarter (2) of a warp per
// leaf; 3: a quarter in the frame pipeline (fewer instructions beside the
// traversal: 0.676 against 0.689 ms per 1080p frame) and a half alone (0.417
// against 0.427 ms).  All forms sum in the same order.
#define FPO_MAT_HALF_WARP 3
#endif
#ifndef FPO_FAST_EXIT
#define FPO_FAST_EXIT 0
#endif
#ifndef FPO_PREFETCH_SIBLINGS
#define FPO_PREFETCH_SIBLINGS 0
#endif

namespace fpo {
namespace {

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

#if FPO_FAST_SIGMOID
// approximate reciprocal (2 ulp): 1 / (1 + e^-x) with e^-x = inf gives 0
__device__ __forceinline__ float sigmoidf_(float x) { return __fdividef(1.0f, 1.0f + __expf(-x)); }
#else
__device__ __forceinline__ float sigmoidf_(float x) { return 1.0f / (1.0f + __expf(-x)); }
#endif

// VW floats from a read-only global address aligned to 4 VW bytes.
template <int VW>
__device__ __forceinline__ void load_vec(const float *p, float *v);

// The FP32 coefficient records of (n1, n2) take 32-byte loads when both
// padded strides are multiples of 8 floats: (31, 5) and (21, 5).
__host__ __device__ constexpr bool fused_ldg256(int n1, int n2)
{
    return ((n1 + 3) & ~3) % 8 == 0 && ((27 * n2 + 3) & ~3) % 8 == 0;
}

// One 32-byte read-only global load (sm_100+ 256-bit vector load); p is
// 32-byte aligned.
__device__ __forceinline__ void ldg256(const float *p, float *v)
{
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
        : "l"(p));
}

template <>
__device__ __forceinline__ void load_vec<8>(const float *p, float *v)
{
    ldg256(p, v);
}

template <>
__device__ __forceinline__ void load_vec<4>(const float *p, float *v)
{
    const float4 w = __ldg(reinterpret_cast<const float4 *>(p));
    v[0] = w.x;
    v[1] = w.y;
    v[2] = w.z;
    v[3] = w.w;
}

}  // namespace

// ---------------------------------------------------------------------------
// Per-frame IDFT table (Eq. 7 and Eq. 9 for every leaf at one time t).
//
// A streaming pass: each CTA walks chunks of MAT_CHUNK leaves.  One thread
// moves a chunk's density records and SH records from HBM into a shared-memory
// stage with two bulk asynchronous copies (completion counted in bytes on the
// stage's mbarrier), keeping `stages` chunks in flight; all threads then form
// the 32-float output records from shared memory, 8 threads per leaf, each
// writing one float4 (coalesced 16-byte stores).

constexpr int MAT_CHUNK = 32;
constexpr int MAT_THREADS = 256;
constexpr int MAT_MAX_STAGES = 6;
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;  // 2 s: a stuck copy, not slowness

// Element i of a stored record in shared memory, as FP32 (storage ST).
template <int ST>
__device__ __forceinline__ float stored(const unsigned char *rec, int i)
{
    if constexpr (ST == FPO_STORAGE_F32) return reinterpret_cast<const float *>(rec)[i];
    else if constexpr (ST == FPO_STORAGE_BF16) return __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(rec)[i]);
    else if constexpr (ST == FPO_STORAGE_F16) return __half2float(reinterpret_cast<const __half *>(rec)[i]);
    else return static_cast<float>(reinterpret_cast<const __nv_fp8_e4m3 *>(rec)[i]);
}

template <int N2, int ST>
__global__ void __launch_bounds__(MAT_THREADS, 8) materialise_kernel(const __grid_constant__ MaterialiseParams p)
{
    extern __shared__ __align__(128) unsigned char mat_smem[];
    __shared__ uint64_t bars[MAT_MAX_STAGES];
    __shared__ uint64_t never;  // FPO_FLAG_TEST_DEVICE_TIMEOUT: a barrier nothing signals
    __shared__ float s_b[MAX_BASIS];
    __shared__ int s_fail;
    const int tid = threadIdx.x;
    const int S = p.stages;
    constexpr uint32_t EB = ST == FPO_STORAGE_F32 ? 4u : (ST == FPO_STORAGE_FP8_E4M3 ? 1u : 2u);
    constexpr bool SCALED = ST == FPO_STORAGE_FP8_E4M3;
    const uint32_t rec_sig = p.sig_stride * EB, rec_z = p.z_stride * EB;  // bytes per leaf
    const uint32_t sig_bytes = MAT_CHUNK * rec_sig;
    const uint32_t z_bytes = MAT_CHUNK * rec_z;
    const uint32_t stage_bytes = sig_bytes + z_bytes + (SCALED ? MAT_CHUNK * 4u : 0u);
    const uint32_t n_chunks = (p.n_leaves + MAT_CHUNK - 1) / MAT_CHUNK;
    const int nb = p.n1 > p.n2 ? p.n1 : p.n2;
    if (tid < nb) s_b[tid] = basis_fp64(tid, p.t, p.period_T);
    if (tid == 0) {
        s_fail = 0;
        for (int s = 0; s < S; ++s) ptx::mbar_init(&bars[s], 1);
        ptx::mbar_init(&never, 1);
        ptx::fence_barrier_init();
    }
    __syncthreads();

    auto issue = [&](uint32_t c, int s) {
        const uint32_t first = c * MAT_CHUNK;
        const uint32_t m = min((uint32_t)MAT_CHUNK, p.n_leaves - first);
        const uint32_t bs = m * rec_sig, bz = m * rec_z;
        unsigned char *dst = mat_smem + (size_t)s * stage_bytes;
        // FP8 scales: 4 bytes per leaf, copied in 16-byte units (the scale
        // array is padded to a multiple of 4 leaves)
        const uint32_t bsc = SCALED ? ((m + 3u) & ~3u) * 4u : 0u;
        ptx::mbar_arrive_expect_tx(&bars[s], bs + bz + bsc);
        ptx::bulk_g2s(dst, static_cast<const unsigned char *>(p.sig) + (size_t)first * rec_sig, bs, &bars[s]);
        ptx::bulk_g2s(dst + sig_bytes, static_cast<const unsigned char *>(p.zc) + (size_t)first * rec_z, bz, &bars[s]);
        if (SCALED) ptx::bulk_g2s(dst + sig_bytes + z_bytes, p.scale + first, bsc, &bars[s]);
    };
    if (tid == 0)
        for (int s = 0; s < S; ++s) {
            const uint32_t c = blockIdx.x + (uint32_t)s * gridDim.x;
            if (c < n_chunks) issue(c, s);
        }

    const int warp = tid >> 5, lane = tid & 31;
    const float b_lane = lane < nb ? s_b[lane] : 0.0f;
    const float b_lo = (lane & 15) < nb ? s_b[lane & 15] : 0.0f;              // half-warp form
    const float b_hi = (lane & 15) + 16 < nb ? s_b[(lane & 15) + 16] : 0.0f;
    float bq[4];                                                             // quarter-warp form
#pragma unroll
    for (int k = 0; k < 4; ++k) bq[k] = (lane & 7) + 8 * k < nb ? s_b[(lane & 7) + 8 * k] : 0.0f;
    float bz[N2 > 0 ? N2 : 1];
#pragma unroll
    for (int i = 0; i < (N2 > 0 ? N2 : 1); ++i) bz[i] = s_b[i];
    uint32_t it = 0;
    for (;; ++it) {
        const uint32_t c = blockIdx.x + it * gridDim.x;
        if (c >= n_chunks) break;
        const int s = (int)(it % (uint32_t)S);
        const uint32_t parity = (it / (uint32_t)S) & 1u;
        // (the failure-path test makes the first wait run out; the drain below
        // still waits for every copy in flight)
        const bool ok = p.test_timeout && it == 0 ? ptx::mbar_wait_bounded(&never, 0, TEST_WAIT_LIMIT_NS)
                                                  : ptx::mbar_wait_bounded(&bars[s], parity, WAIT_LIMIT_NS);
        if (!ok) s_fail = 1;
        __syncthreads();
        if (s_fail) break;
        const uint32_t first = c * MAT_CHUNK;
        const int m = (int)min((uint32_t)MAT_CHUNK, p.n_leaves - first);
        const unsigned char *stage_sig = mat_smem + (size_t)s * stage_bytes;
        const unsigned char *stage_z = stage_sig + sig_bytes;
        const float *stage_scale = reinterpret_cast<const float *>(stage_z + z_bytes);
        if constexpr ((FPO_MAT_HALF_WARP == 2 || FPO_MAT_HALF_WARP == 3) && N2 == 5 && ST == FPO_STORAGE_F32) {
            if (!p.half_table && (FPO_MAT_HALF_WARP == 2 || p.pipeline)) {
                // A quarter warp (8 lanes) per leaf, four leaves per pass:
                // lane ql forms the products of i = ql, ql + 8, ql + 16,
                // ql + 24 and sums them as the full warp's butterfly does
                // ((i, i + 16), then + (i + 8, i + 24)), then xor 4, 2, 1 within
                // the quarter; it forms z_{ql + 8k}, k = 0..3, and stores
                // row[ql + 8k].
                const int qw = lane >> 3, ql = lane & 7;
                for (int l0 = 4 * warp; l0 < m; l0 += 4 * (MAT_THREADS / 32)) {
                    const int l = l0 + qw;
                    const bool valid = l < m;
                    const float *sg = reinterpret_cast<const float *>(stage_sig + (valid ? l : l0) * rec_sig);
                    const float *zz = reinterpret_cast<const float *>(stage_z + (valid ? l : l0) * rec_z);
                    float pr[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) pr[k] = ql + 8 * k < p.n1 ? __fmul_rn(sg[ql + 8 * k], bq[k]) : 0.0f;
                    float part = __fadd_rn(__fadd_rn(pr[0], pr[2]), __fadd_rn(pr[1], pr[3]));
#pragma unroll
                    for (int o = 4; o >= 1; o >>= 1) part = __fadd_rn(part, __shfl_xor_sync(0xffffffffu, part, o));
                    float zq[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        zq[k] = 0.0f;
                        if (ql + 8 * k < 27) {
#pragma unroll
                            for (int i = 0; i < 5; ++i) zq[k] = fmaf(zz[(ql + 8 * k) * 5 + i], bz[i], zq[k]);
                        }
                    }
                    float o[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        // row[ql + 8k] = z[ql + 8k - 1]: lane ql - 1's zq[k], or lane 7's zq[k - 1] for ql = 0
                        const float up = __shfl_up_sync(0xffffffffu, zq[k], 1, 8);
                        const float from7 = __shfl_sync(0xffffffffu, zq[k > 0 ? k - 1 : 0], 7, 8);
                        const int j = ql + 8 * k;
                        o[k] = ql == 0 ? (k == 0 ? fmaxf(part, 0.0f) : from7) : (j <= 27 ? up : 0.0f);
                    }
                    if (valid) {
                        float *row = p.table + ((size_t)first + l) * TABLE_STRIDE;
#pragma unroll
                        for (int k = 0; k < 4; ++k) row[ql + 8 * k] = o[k];
                    }
                }
                __syncthreads();  // every thread is done with stage s
                if (tid == 0) {
                    const uint32_t c2 = c + (uint32_t)S * gridDim.x;
                    if (c2 < n_chunks) issue(c2, s);
                }
                continue;
            }
        }
        if constexpr ((FPO_MAT_HALF_WARP == 1 || FPO_MAT_HALF_WARP == 3) && N2 == 5 && ST == FPO_STORAGE_F32) {
            if (!p.half_table) {
                // Half a warp per leaf, two leaves per pass: lane sl of a half
                // forms k_sl b_sl + k_{sl+16} b_{sl+16} (the first step of the
                // full warp's butterfly) and the butterfly continues within the
                // half, so the density sums in the same order; z_{sl} and
                // z_{sl+16} are the same sequential sums.  Each lane stores
                // row[sl] and row[sl + 16].
                const int hw = lane >> 4, sl = lane & 15;
                for (int l0 = 2 * warp; l0 < m; l0 += 2 * (MAT_THREADS / 32)) {
                    const int l = l0 + hw;
                    const bool valid = l < m;
                    const float *sg = reinterpret_cast<const float *>(stage_sig + (valid ? l : l0) * rec_sig);
                    const float *zz = reinterpret_cast<const float *>(stage_z + (valid ? l : l0) * rec_z);
                    const float p1 = sl < p.n1 ? __fmul_rn(sg[sl], b_lo) : 0.0f;
                    const float p2 = sl + 16 < p.n1 ? __fmul_rn(sg[sl + 16], b_hi) : 0.0f;
                    float part = __fadd_rn(p1, p2);
#pragma unroll
                    for (int o = 8; o >= 1; o >>= 1) part = __fadd_rn(part, __shfl_xor_sync(0xffffffffu, part, o));
                    float za = 0.0f, zb = 0.0f;
#pragma unroll
                    for (int i = 0; i < 5; ++i) za = fmaf(zz[sl * 5 + i], bz[i], za);
                    if (sl < 11) {
#pragma unroll
                        for (int i = 0; i < 5; ++i) zb = fmaf(zz[(sl + 16) * 5 + i], bz[i], zb);
                    }
                    const float za_prev = __shfl_up_sync(0xffffffffu, za, 1, 16);
                    const float zb_prev = __shfl_up_sync(0xffffffffu, zb, 1, 16);
                    const float za_15 = __shfl_sync(0xffffffffu, za, 15, 16);
                    const float o1 = sl == 0 ? fmaxf(part, 0.0f) : za_prev;
                    const float o2 = sl == 0 ? za_15 : (sl + 16 <= 27 ? zb_prev : 0.0f);
                    if (valid) {
                        float *row = p.table + ((size_t)first + l) * TABLE_STRIDE;
                        row[sl] = o1;
                        row[sl + 16] = o2;
                    }
                }
                __syncthreads();  // every thread is done with stage s
                if (tid == 0) {
                    const uint32_t c2 = c + (uint32_t)S * gridDim.x;
                    if (c2 < n_chunks) issue(c2, s);
                }
                continue;
            }
        }
        // One warp per leaf: lane i < n1 forms k_sigma_i b_i and a butterfly
        // sums the density; lanes 0..26 form z_{lane}(t) from n2 consecutive
        // elements.  Lane j then stores output j.
        for (int l = warp; l < m; l += MAT_THREADS / 32) {
            const unsigned char *sg = stage_sig + l * rec_sig;
            const unsigned char *zz = stage_z + l * rec_z;
            float part = lane < p.n1 ? stored<ST>(sg, lane) * b_lane : 0.0f;
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            float v = 0.0f;
            if (lane < 27) {
                if constexpr (N2 > 0) {
#pragma unroll
                    for (int i = 0; i < N2; ++i) v = fmaf(stored<ST>(zz, lane * N2 + i), bz[i], v);
                } else {
                    for (int i = 0; i < p.n2; ++i) v = fmaf(stored<ST>(zz, lane * p.n2 + i), s_b[i], v);
                }
            }
            if (SCALED) {
                const float sc = stage_scale[l];
                part *= sc;
                v *= sc;
            }
            const float zprev = __shfl_up_sync(0xffffffffu, v, 1);
            const float outv = lane == 0 ? fmaxf(part, 0.0f) : (lane <= 27 ? zprev : 0.0f);
            if (p.half_table)
                reinterpret_cast<__half *>(p.table)[((size_t)first + l) * TABLE_STRIDE + lane] = __float2half_rn(outv);
            else
                p.table[((size_t)first + l) * TABLE_STRIDE + lane] = outv;
        }
        __syncthreads();  // every thread is done with stage s
        if (tid == 0) {
            const uint32_t c2 = c + (uint32_t)S * gridDim.x;
            if (c2 < n_chunks) issue(c2, s);
        }
    }
    if (s_fail && tid == 0) {
        // Drain the copies still in flight (bounded), then report.
        for (uint32_t k = it; k < it + (uint32_t)S; ++k) {
            const uint32_t c = blockIdx.x + k * gridDim.x;
            if (c >= n_chunks) break;
            ptx::mbar_wait_bounded(&bars[k % (uint32_t)S], (k / (uint32_t)S) & 1u, WAIT_LIMIT_NS);
        }
        atomicOr(p.status, STATUS_DEVICE_TIMEOUT);
    }
}

// Reduced-precision storages (BF16, FP16, FP8) with n2 = 5: the pass is
// bound by instructions, not bytes, in the warp-per-leaf form above (77 warp
// instructions per leaf, shared-memory bank conflicts on 2-byte elements).
// Here one thread owns one leaf of a 256-leaf chunk: 16-byte loads of its
// records from the same bulk-copy ring, unpacked in registers, the density
// products summed in the same tree order as the warp's butterfly and each z
// accumulated in the same order as above, so both kernels give the same
// bits; the row is written with 16-byte stores.
// One CTA per SM with 256-leaf stages on its own; 128-leaf stages when it
// shares the SM with the traversal (frame pipeline).
constexpr int ML_CHUNK = 256, ML_CHUNK_PIPE = 128, ML_N2 = 5;

// The 16 bytes of w as FP32 values (4 for FP32 storage, 8 for 16-bit, 16 for FP8).
template <int ST>
__device__ __forceinline__ void unpack16(const uint4 w, float *v)
{
    const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if constexpr (ST == FPO_STORAGE_F32) {
            v[k] = __uint_as_float(u[k]);
        } else if constexpr (ST == FPO_STORAGE_BF16) {
            v[2 * k] = __uint_as_float(u[k] << 16);
            v[2 * k + 1] = __uint_as_float(u[k] & 0xffff0000u);
        } else if constexpr (ST == FPO_STORAGE_F16) {
            const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&u[k]));
            v[2 * k] = f.x;
            v[2 * k + 1] = f.y;
        } else {
            const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(u[k] & 0xffffu), __NV_E4M3);
            const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(u[k] >> 16), __NV_E4M3);
            const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&lo));
            const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&hi));
            v[4 * k] = a.x;
            v[4 * k + 1] = a.y;
            v[4 * k + 2] = b.x;
            v[4 * k + 3] = b.y;
        }
    }
}

template <int ST, int CH>
__global__ void __launch_bounds__(CH, ST == FPO_STORAGE_F32 ? 4 : 1) materialise_leaf_kernel(const __grid_constant__ MaterialiseParams p)
{
    extern __shared__ __align__(128) unsigned char mat_smem[];
    __shared__ uint64_t bars[MAT_MAX_STAGES];
    __shared__ uint64_t never;  // FPO_FLAG_TEST_DEVICE_TIMEOUT: a barrier nothing signals
    __shared__ float s_b[MAX_BASIS];
    __shared__ int s_fail;
    const int tid = threadIdx.x;
    const int S = p.stages;
    constexpr uint32_t EB = ST == FPO_STORAGE_F32 ? 4u : (ST == FPO_STORAGE_FP8_E4M3 ? 1u : 2u);
    constexpr int PER = 16 / (int)EB;              // elements per 16-byte load
    constexpr bool SCALED = ST == FPO_STORAGE_FP8_E4M3;
    constexpr int SIG_ELEMS = 32;                  // n1 <= 32, padded to 16 bytes
    constexpr int Z_ELEMS = (27 * ML_N2 + PER - 1) / PER * PER;
    const uint32_t rec_sig = SIG_ELEMS * EB, rec_z = Z_ELEMS * EB;
    const uint32_t sig_bytes = CH * rec_sig, z_bytes = CH * rec_z;
    const uint32_t stage_bytes = sig_bytes + z_bytes + (SCALED ? CH * 4u : 0u);
    const uint32_t n_chunks = (p.n_leaves + CH - 1) / CH;
    const int nb = p.n1 > ML_N2 ? p.n1 : ML_N2;
    if (tid < MAX_BASIS) s_b[tid] = tid < nb ? basis_fp64(tid, p.t, p.period_T) : 0.0f;
    if (tid == 0) {
        s_fail = 0;
        for (int s = 0; s < S; ++s) ptx::mbar_init(&bars[s], 1);
        ptx::mbar_init(&never, 1);
        ptx::fence_barrier_init();
    }
    __syncthreads();
    // Beside the traversal (frame pipeline) the records, read once, are
    // marked for early eviction from L2, which leaves more of it to the
    // traversal's nodes and table lines (measured: 0.580 against 0.588 ms per
    // BF16 frame; the FP32 pass, in the warp-cooperative form, gains nothing).
    const bool hint_ld = p.pipeline != 0;
    const uint64_t pol = ptx::l2_evict_first();
    auto copy = [&](void *d, const void *src, uint32_t n, uint64_t *b) {
        if (hint_ld) ptx::bulk_g2s_hint(d, src, n, b, pol);
        else ptx::bulk_g2s(d, src, n, b);
    };
    auto issue = [&](uint32_t c, int s) {
        const uint32_t first = c * CH;
        const uint32_t m = min((uint32_t)CH, p.n_leaves - first);
        unsigned char *dst = mat_smem + (size_t)s * stage_bytes;
        const uint32_t bsc = SCALED ? ((m + 3u) & ~3u) * 4u : 0u;
        ptx::mbar_arrive_expect_tx(&bars[s], m * rec_sig + m * rec_z + bsc);
        copy(dst, static_cast<const unsigned char *>(p.sig) + (size_t)first * rec_sig, m * rec_sig, &bars[s]);
        copy(dst + sig_bytes, static_cast<const unsigned char *>(p.zc) + (size_t)first * rec_z, m * rec_z, &bars[s]);
        if (SCALED) copy(dst + sig_bytes + z_bytes, p.scale + first, bsc, &bars[s]);
    };
    if (tid == 0)
        for (int s = 0; s < S; ++s) {
            const uint32_t c = blockIdx.x + (uint32_t)s * gridDim.x;
            if (c < n_chunks) issue(c, s);
        }
    float b[SIG_ELEMS], bz[ML_N2];
#pragma unroll
    for (int i = 0; i < SIG_ELEMS; ++i) b[i] = i < p.n1 ? s_b[i] : 0.0f;
#pragma unroll
    for (int i = 0; i < ML_N2; ++i) bz[i] = s_b[i];
    uint32_t it = 0;
    for (;; ++it) {
        const uint32_t c = blockIdx.x + it * gridDim.x;
        if (c >= n_chunks) break;
        const int s = (int)(it % (uint32_t)S);
        const uint32_t parity = (it / (uint32_t)S) & 1u;
        // (the failure-path test makes the first wait run out; the drain below
        // still waits for every copy in flight)
        const bool ok = p.test_timeout && it == 0 ? ptx::mbar_wait_bounded(&never, 0, TEST_WAIT_LIMIT_NS)
                                                  : ptx::mbar_wait_bounded(&bars[s], parity, WAIT_LIMIT_NS);
        if (!ok) s_fail = 1;
        __syncthreads();
        if (s_fail) break;
        const uint32_t first = c * CH;
        const int m = (int)min((uint32_t)CH, p.n_leaves - first);
        const unsigned char *stage = mat_smem + (size_t)s * stage_bytes;
        if (tid < m) {
            const uint4 *sg = reinterpret_cast<const uint4 *>(stage + tid * rec_sig);
            const uint4 *zz = reinterpret_cast<const uint4 *>(stage + sig_bytes + tid * rec_z);
            // density: products k_i b_i, summed as the warp butterfly does
            // (pairs i, i + 16, then i, i + 8, ... down to i, i + 1)
            float part[SIG_ELEMS];
#pragma unroll
            for (int k = 0; k < SIG_ELEMS / PER; ++k) {
                float v[PER];
                unpack16<ST>(sg[k], v);
#pragma unroll
                for (int j = 0; j < PER; ++j) part[k * PER + j] = __fmul_rn(v[j], b[k * PER + j]);
            }
            // (_rn: no contraction of a product into the sums, as across lanes)
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1)
#pragma unroll
                for (int i = 0; i < o; ++i) part[i] = __fadd_rn(part[i], part[i + o]);
            float z[27];
#pragma unroll
            for (int q = 0; q < 27; ++q) z[q] = 0.0f;
#pragma unroll
            for (int k = 0; k < Z_ELEMS / PER; ++k) {
                float v[PER];
                unpack16<ST>(zz[k], v);
#pragma unroll
                for (int j = 0; j < PER; ++j) {
                    const int e = k * PER + j;
                    if (e < 27 * ML_N2) z[e / ML_N2] = fmaf(v[j], bz[e % ML_N2], z[e / ML_N2]);
                }
            }
            float sigma = part[0];
            if (SCALED) {
                const float sc = reinterpret_cast<const float *>(stage + sig_bytes + z_bytes)[tid];
                sigma *= sc;
#pragma unroll
                for (int q = 0; q < 27; ++q) z[q] *= sc;
            }
            sigma = fmaxf(sigma, 0.0f);
            const size_t leaf = (size_t)first + tid;
            if (p.half_table) {
                uint32_t h[16];
                {
                    const __half2 hh = __floats2half2_rn(sigma, z[0]);
                    h[0] = *reinterpret_cast<const uint32_t *>(&hh);
                }
#pragma unroll
                for (int q = 1; q < 14; ++q) {
                    const __half2 hh = __floats2half2_rn(z[2 * q - 1], z[2 * q]);
                    h[q] = *reinterpret_cast<const uint32_t *>(&hh);
                }
                h[14] = h[15] = 0u;
                uint4 *dst = reinterpret_cast<uint4 *>(reinterpret_cast<__half *>(p.table) + leaf * TABLE_STRIDE);
#pragma unroll
                for (int q = 0; q < 4; ++q) dst[q] = make_uint4(h[4 * q], h[4 * q + 1], h[4 * q + 2], h[4 * q + 3]);
            } else {
                float4 *dst = reinterpret_cast<float4 *>(p.table + leaf * TABLE_STRIDE);
                dst[0] = make_float4(sigma, z[0], z[1], z[2]);
#pragma unroll
                for (int q = 1; q < 7; ++q) dst[q] = make_float4(z[4 * q - 1], z[4 * q], z[4 * q + 1], z[4 * q + 2]);
                dst[7] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
        }
        __syncthreads();  // every thread is done with stage s
        if (tid == 0) {
            const uint32_t c2 = c + (uint32_t)S * gridDim.x;
            if (c2 < n_chunks) issue(c2, s);
        }
    }
    if (s_fail && tid == 0) {
        for (uint32_t k = it; k < it + (uint32_t)S; ++k) {
            const uint32_t c = blockIdx.x + k * gridDim.x;
            if (c >= n_chunks) break;
            ptx::mbar_wait_bounded(&bars[k % (uint32_t)S], (k / (uint32_t)S) & 1u, WAIT_LIMIT_NS);
        }
        atomicOr(p.status, STATUS_DEVICE_TIMEOUT);
    }
}

// The thread-per-leaf form applies to the reduced-precision storages with
// n2 = 5 and density records of 32 elements (n1 from 25 or, for FP8, 17 up
// to 32).  FPO_PIPE_F32_LEAF 1 also uses it for FP32 records in the frame
// pipeline (measured slower: its 172 KB ring leaves the traversal 28 KB of
// L1, and four warps do not keep up).
#ifndef FPO_PIPE_F32_LEAF
#define FPO_PIPE_F32_LEAF 0
#endif
static bool leaf_form(int storage, int n1, int n2, bool pipe = false)
{
    const bool f32 = storage == FPO_STORAGE_F32 && pipe && FPO_PIPE_F32_LEAF;
    if (!f32 && (storage < FPO_STORAGE_BF16 || storage > FPO_STORAGE_FP8_E4M3)) return false;
    if (n2 != ML_N2 || n1 < 1 || n1 > 32) return false;
    const RecordLayout L = record_layout(storage, n1, n2);  // the kernel's fixed record strides
    const int per = 16 / L.elem_bytes;
    return L.sig_elems == 32 && L.z_elems == (27 * ML_N2 + per - 1) / per * per;
}

int materialise_stages(int storage, int n1, int n2)
{
    const RecordLayout L = record_layout(storage, n1, n2);
    if (leaf_form(storage, n1, n2)) {  // one CTA per SM, 256 leaves per stage
        const int stage = ML_CHUNK * (L.sig_bytes() + L.z_bytes() + (L.scaled ? 4 : 0));
        int s = (200 * 1024) / stage;
        if (s > MAT_MAX_STAGES) s = MAT_MAX_STAGES;
        if (s < 2) s = 2;
        return s;
    }
    const int stage = MAT_CHUNK * (L.sig_bytes() + L.z_bytes() + (L.scaled ? 4 : 0));
    int s = (100 * 1024) / stage;  // two CTAs per SM
    if (s > MAT_MAX_STAGES) s = MAT_MAX_STAGES;
    if (s < 2) s = 2;
    return s;
}

static int record_bytes(int storage, int n1, int n2)
{
    const RecordLayout L = record_layout(storage, n1, n2);
    return L.sig_bytes() + L.z_bytes() + (L.scaled ? 4 : 0);
}

static int clamp_stages(int s)
{
    return s > MAT_MAX_STAGES ? MAT_MAX_STAGES : (s < 2 ? 2 : s);
}

MatShape materialise_pipeline_shape(int storage, int n1, int n2, int smem_budget)
{
    MatShape m{};
    if (leaf_form(storage, n1, n2, true)) {  // one CTA of ML_CHUNK_PIPE threads
        const int stage = ML_CHUNK_PIPE * record_bytes(storage, n1, n2);
        m.ctas_per_sm = 1;
        m.stages = clamp_stages(smem_budget / stage);
        m.smem_per_cta = m.stages * stage;
    } else {  // two CTAs of the warp-cooperative form
        const int stage = MAT_CHUNK * record_bytes(storage, n1, n2);
        m.ctas_per_sm = 2;
        m.stages = clamp_stages(smem_budget / 2 / stage);
        m.smem_per_cta = m.stages * stage;
    }
    return m;
}

// Leaves per stage (= threads of the thread-per-leaf form); 0 for the
// warp-cooperative form.
static int leaf_chunk(const MaterialiseParams &p)
{
    if (!leaf_form(p.storage, p.n1, p.n2, p.pipeline != 0)) return 0;
    return p.pipeline ? ML_CHUNK_PIPE : ML_CHUNK;
}

int materialise_smem_bytes(const MaterialiseParams &p)
{
    const int lc = leaf_chunk(p);
    return p.stages * (lc ? lc : MAT_CHUNK) * record_bytes(p.storage, p.n1, p.n2);
}

template <int CH>
static void *pick_leaf(int storage)
{
    switch (storage) {
    case FPO_STORAGE_F32: return (void *)materialise_leaf_kernel<FPO_STORAGE_F32, ML_CHUNK_PIPE>;
    case FPO_STORAGE_BF16: return (void *)materialise_leaf_kernel<FPO_STORAGE_BF16, CH>;
    case FPO_STORAGE_F16: return (void *)materialise_leaf_kernel<FPO_STORAGE_F16, CH>;
    default: return (void *)materialise_leaf_kernel<FPO_STORAGE_FP8_E4M3, CH>;
    }
}

template <int N2>
static void *pick_materialise(int storage)
{
    switch (storage) {
    case FPO_STORAGE_BF16: return (void *)materialise_kernel<N2, FPO_STORAGE_BF16>;
    case FPO_STORAGE_F16: return (void *)materialise_kernel<N2, FPO_STORAGE_F16>;
    case FPO_STORAGE_FP8_E4M3: return (void *)materialise_kernel<N2, FPO_STORAGE_FP8_E4M3>;
    default: return (void *)materialise_kernel<N2, FPO_STORAGE_F32>;
    }
}

int launch_materialise(const MaterialiseParams &p, int sm_count, void *stream)
{
    if (p.n_leaves == 0) return (int)cudaSuccess;
    if (p.storage < FPO_STORAGE_F32 || p.storage > FPO_STORAGE_FP8_E4M3 || !p.sig || !p.zc)
        return (int)cudaErrorInvalidValue;  // no coefficient records (e.g. LATENT storage)
    const int lc = leaf_chunk(p);
    const bool lf = lc > 0;
    const int chunk = lf ? lc : MAT_CHUNK;
    const int threads = lf ? lc : MAT_THREADS;
    const int smem = materialise_smem_bytes(p);
    const void *kern;
    if (lf)
        kern = lc == ML_CHUNK ? pick_leaf<ML_CHUNK>(p.storage) : pick_leaf<ML_CHUNK_PIPE>(p.storage);
    else
        kern = p.n2 == 5 ? pick_materialise<5>(p.storage)
                         : (p.n2 == 11 ? pick_materialise<11>(p.storage) : pick_materialise<0>(p.storage));
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 p.carveout > 0 ? p.carveout : (int)cudaSharedmemCarveoutDefault);
    if (e != cudaSuccess) return (int)e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return (int)e;
    if (per_sm < 1) per_sm = 1;
    if (p.max_ctas_per_sm > 0 && per_sm > p.max_ctas_per_sm) per_sm = p.max_ctas_per_sm;
    const uint32_t n_chunks = (p.n_leaves + chunk - 1) / chunk;
    uint64_t blocks = (uint64_t)sm_count * per_sm;
    if (blocks > n_chunks) blocks = n_chunks;
    void *args[] = {(void *)&p};
    e = cudaLaunchKernel(kern, dim3((unsigned)blocks), dim3(threads), args, smem,
                         (cudaStream_t)stream);
    if (e != cudaSuccess) return (int)e;
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

// Per-lane state of one ray, kept in registers across the warp's step loop.
struct RayState {
    float go[3];   // origin in grid units, moved to the cube entry point
    float gd[3];   // direction in grid units
    float inv[3];  // 1 / gd, 0 where gd == 0
    int pos[3];    // 1 where gd > 0: exit plane = lo + pos * size
    int zmask;     // bit a set where gd[a] == 0 (that axis is never crossed)
    float Y[9];    // real SH of the unit direction (Eq. 1)
    float C0, C1, C2, T, t;
    int P[3];      // finest-level cell holding the current point
    int lvl_start; // deepest ancestor level valid in the per-thread stack
    uint32_t steps, n_visits, ray;
};


__device__ __forceinline__ void write_result(const TraverseParams &p, const RayState &R, bool dbg)
{
    p.out_rgb[3 * (size_t)R.ray] = fmaf(R.T, p.bg[0], R.C0);
    p.out_rgb[3 * (size_t)R.ray + 1] = fmaf(R.T, p.bg[1], R.C1);
    p.out_rgb[3 * (size_t)R.ray + 2] = fmaf(R.T, p.bg[2], R.C2);
    if (dbg) {
        if (p.flags & FPO_FLAG_OUT_T) p.out_T[R.ray] = R.T;
        if (p.flags & FPO_FLAG_RECORD_VISITS) p.visit_count[R.ray] = R.n_visits;
    }
}

// Sets up ray `ray` (camera pixel (px, py) or explicit ray): generation,
// SH basis, clip against the grid cube.  Returns false when the ray misses
// the tree (its background result is written at once).
__device__ bool init_ray_geom(const TraverseParams &p, const FrameShared &fs, bool prt, float *s_bray,
                              int stride, uint32_t *s_stack, RayState &R, uint32_t ray, int px, int py)
{
    float ox, oy, oz, dx, dy, dz;
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
        ox = p.fr.ro[3 * (size_t)ray];
        oy = p.fr.ro[3 * (size_t)ray + 1];
        oz = p.fr.ro[3 * (size_t)ray + 2];
        dx = p.fr.rd[3 * (size_t)ray];
        dy = p.fr.rd[3 * (size_t)ray + 1];
        dz = p.fr.rd[3 * (size_t)ray + 2];
    }
    {
        const float inv = 1.0f / sqrtf(dx * dx + dy * dy + dz * dz);
        dx *= inv;
        dy *= inv;
        dz *= inv;
    }
    if (prt) {
        // Eq. 8 at this ray's own time, one column of the per-thread table
        const float u = p.fr.rt[ray] / (float)p.fr.period_T;
        const int nb = p.n1 > p.n2 ? p.n1 : p.n2;
        for (int i = 0; i < nb; ++i) s_bray[i * stride] = basis_fp32(i, u);
    }
    sh_basis(dx, dy, dz, R.Y);
    R.C0 = R.C1 = R.C2 = 0.0f;
    R.T = 1.0f;
    R.t = 0.0f;
    R.steps = 0;
    R.n_visits = 0;
    R.ray = ray;
    R.lvl_start = 0;

    const int G = 1 << p.depth;
    const float gs = p.grid_scale;
    R.go[0] = (ox - p.amin[0]) * gs;
    R.go[1] = (oy - p.amin[1]) * gs;
    R.go[2] = (oz - p.amin[2]) * gs;
    R.gd[0] = dx * gs;
    R.gd[1] = dy * gs;
    R.gd[2] = dz * gs;
    float t0 = 0.0f, t1 = FLT_MAX;
    bool hit = p.root_kind != ROOT_EMPTY;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (R.gd[a] != 0.0f) {
            R.inv[a] = 1.0f / R.gd[a];
            const float ta = (0.0f - R.go[a]) * R.inv[a], tb = ((float)G - R.go[a]) * R.inv[a];
            t0 = fmaxf(t0, fminf(ta, tb));
            t1 = fminf(t1, fmaxf(ta, tb));
        } else {
            R.inv[a] = 0.0f;
            if (R.go[a] < 0.0f || R.go[a] > (float)G) hit = false;
        }
    }
    if (!(hit && t0 < t1)) return false;
    // Distances are measured from the entry point from here on.
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        R.go[a] = fmaf(t0, R.gd[a], R.go[a]);
        R.P[a] = min(max((int)floorf(R.go[a]), 0), G - 1);
        R.pos[a] = R.gd[a] > 0.0f ? 1 : 0;
    }
    R.zmask = (R.gd[0] == 0.0f ? 1 : 0) | (R.gd[1] == 0.0f ? 2 : 0) | (R.gd[2] == 0.0f ? 4 : 0);
    s_stack[0] = 0;
    return true;
}

// As init_ray_geom; a ray that misses the tree gets its background result.
template <bool DBG>
__device__ __forceinline__ bool init_ray(const TraverseParams &p, const FrameShared &fs, bool prt,
                                         float *s_bray, int stride, uint32_t *s_stack, RayState &R,
                                         uint32_t ray, int px, int py)
{
    if (init_ray_geom(p, fs, prt, s_bray, stride, s_stack, R, ray, px, py)) return true;
    write_result(p, R, DBG);
    return false;
}

// The cube holding cell R.P: its kind (ROOT_EMPTY / ROOT_LEAF), leaf index and
// level.  Descends from the deepest still-valid ancestor in the per-thread
// stack, updating the stack on the way down.
struct Cube {
    uint32_t kind, leaf;
    int lvl;
};

__device__ __forceinline__ Cube locate(const TraverseParams &p, const uint32_t *__restrict__ s_nodes,
                                       uint32_t *s_stack, int stride, const int P[3], int lvl_start)
{
    Cube cb;
    cb.leaf = 0;
    if (p.root_kind == ROOT_LEAF) {
        cb.lvl = 0;
        cb.kind = ROOT_LEAF;
        return cb;
    }
    const int D = p.depth;
    int lvl = lvl_start;
    uint32_t node = s_stack[lvl * stride];
    for (;;) {
        const int sh = D - 1 - lvl;
        const uint32_t c = ((P[0] >> sh) & 1) | (((P[1] >> sh) & 1) << 1) | (((P[2] >> sh) & 1) << 2);
        const uint32_t idx = node * 8 + c;
#if FPO_NODE_SMEM == 0
        // every node slot from global memory (read-only path)
        const uint32_t sl = __ldg(p.nodes + idx);
        (void)s_nodes;
#elif FPO_GENERIC_NODE_LOAD
        // one generic load from shared (top nodes) or global memory: no branch
        // between two load paths for lanes at different levels
        const uint32_t *src = node < p.n_smem_nodes ? s_nodes : p.nodes;
        const uint32_t sl = src[idx];
#else
        const uint32_t sl = node < p.n_smem_nodes ? s_nodes[idx] : __ldg(p.nodes + idx);
#endif
        ++lvl;
        if (sl == 0u) { cb.kind = ROOT_EMPTY; break; }
        if (sl & LEAF_BIT) { cb.kind = ROOT_LEAF; cb.leaf = sl & ~LEAF_BIT; break; }
        node = sl;
        s_stack[lvl * stride] = node;
    }
    cb.lvl = lvl;
    return cb;
}

// Exit of cube (level lvl, 2^(D - lvl) finest cells a side) holding R.P:
// the exit distance tx along the ray, the exit axis m (ties: x < y < z) and
// the cube's lower corner lo.
__device__ __forceinline__ float cube_exit(const RayState &R, int D, int lvl, int &m, int lo[3], int &csz)
{
    float te[3];
    if (FPO_FAST_EXIT && lvl == D) {
        // a finest cell: the same planes as below with csz = 1, lo = P
        csz = 1;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = R.P[a];
            te[a] = (R.zmask >> a) & 1 ? FLT_MAX : ((float)(R.P[a] + R.pos[a]) - R.go[a]) * R.inv[a];
        }
    } else {
        csz = 1 << (D - lvl);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = R.P[a] & ~(csz - 1);
            // (plane - go) is exact for nearby planes (Sterbenz), so te carries
            // one rounding of the product
            te[a] = (R.zmask >> a) & 1 ? FLT_MAX : ((float)(lo[a] + R.pos[a] * csz) - R.go[a]) * R.inv[a];
        }
    }
    m = 0;
    float tx = te[0];
    if (te[1] < tx) { tx = te[1]; m = 1; }
    if (te[2] < tx) { tx = te[2]; m = 2; }
    return tx;
}

// Next cell after leaving the cube through axis m at distance tx.  Along m:
// the adjacent cube; along the other axes: the cell holding the exit point,
// clamped to this cube's extent and never moving backwards, so every step
// makes progress.  A finest-level cube keeps the other two coordinates.
// Returns false when the ray leaves the grid.
__device__ __forceinline__ bool next_cell(const RayState &R, int G, int m, const int lo[3], int csz,
                                          float tx, int Pn[3])
{
    bool inside = true;
    if (FPO_FAST_STEP && csz == 1) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            Pn[a] = R.P[a];
            if (a == m) {
                Pn[a] += 2 * R.pos[a] - 1;
                inside = (unsigned)Pn[a] < (unsigned)G;
            }
        }
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (a == m) {
                Pn[a] = R.pos[a] ? lo[a] + csz : lo[a] - 1;
                inside = (unsigned)Pn[a] < (unsigned)G;
            } else {
                int q = (int)floorf(fmaf(tx, R.gd[a], R.go[a]));
                q = min(max(q, lo[a]), lo[a] + csz - 1);
                if (R.gd[a] > 0.0f) q = max(q, R.P[a]);
                else if (R.gd[a] < 0.0f) q = min(q, R.P[a]);
                Pn[a] = q;
            }
        }
    }
    return inside;
}

// Moves R to cell Pn: the deepest common ancestor level of the old and the
// new cell becomes the next descent's starting level.
__device__ __forceinline__ void move_to(RayState &R, int D, const int Pn[3], float tx)
{
    R.t = fmaxf(R.t, tx);
    const uint32_t diff = (uint32_t)((R.P[0] ^ Pn[0]) | (R.P[1] ^ Pn[1]) | (R.P[2] ^ Pn[2]));
    R.lvl_start = D - 1 - (31 - __clz(diff));
    R.P[0] = Pn[0];
    R.P[1] = Pn[1];
    R.P[2] = Pn[2];
}

// Table modes of the traversal: the fused per-visit IDFT, or the per-frame
// table in FP32 (128-byte lines) or FP16 (64-byte lines).
constexpr int TM_FUSED = 0, TM_TABLE_F32 = 1, TM_TABLE_F16 = 2;

__device__ __forceinline__ const float4 *table_record(const TraverseParams &p, uint32_t leaf)
{
    return p.table + (size_t)leaf * (TABLE_STRIDE / 4);
}

__device__ __forceinline__ const __half *table_record_f16(const TraverseParams &p, uint32_t leaf)
{
    return reinterpret_cast<const __half *>(p.table) + (size_t)leaf * TABLE_STRIDE;
}

// Shades one leaf segment of length delta (Eq. 7 and 9 from the table or
// fused, Eq. 1 colour, emission-absorption update).  Returns true when the
// transmittance fell below stop_T.
template <int TM, bool DBG, int N1, int N2>
__device__ __forceinline__ bool shade(const TraverseParams &p, const float *bsrc, int bstride,
                                      RayState &R, uint32_t leaf, float delta)
{
    float sigma, z[27];
    if constexpr (TM == TM_TABLE_F16) {
        // the 64-byte FP16 line: two 32-byte loads, widened to FP32
        const float *hrec = reinterpret_cast<const float *>(table_record_f16(p, leaf));
        float raw[16], v[32];
        ldg256(hrec, raw);
        ldg256(hrec + 8, raw + 8);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&raw[q]));
            v[2 * q] = f.x;
            v[2 * q + 1] = f.y;
        }
        sigma = v[0];
#pragma unroll
        for (int q = 0; q < 27; ++q) z[q] = v[q + 1];
    } else if constexpr (TM == TM_TABLE_F32) {
        const float4 *rec = table_record(p, leaf);
        float v[32];
#if FPO_LDG256
        // the 112 used bytes of the 128-byte table line: three 32-byte loads
        // and one 16-byte load (half the load instructions, and half the L1
        // wavefronts, of 16-byte loads; no registers for the padding)
#pragma unroll
        for (int q = 0; q < 3; ++q) ldg256(reinterpret_cast<const float *>(rec) + 8 * q, v + 8 * q);
        {
            const float4 w = __ldg(rec + 6);
            v[24] = w.x;
            v[25] = w.y;
            v[26] = w.z;
            v[27] = w.w;
        }
#else
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            const float4 w = __ldg(rec + q);
            v[4 * q] = w.x;
            v[4 * q + 1] = w.y;
            v[4 * q + 2] = w.z;
            v[4 * q + 3] = w.w;
        }
#endif
        sigma = v[0];
#pragma unroll
        for (int q = 0; q < 27; ++q) z[q] = v[q + 1];
    } else {
        const float4 *sr = p.sig + (size_t)leaf * p.sig_stride4;
        const float *zr = p.zc + (size_t)leaf * p.z_stride;
        float bz[N2];
#pragma unroll
        for (int i = 0; i < N2; ++i) bz[i] = bsrc[i * bstride];
#pragma unroll
        for (int q = 0; q < 27; ++q) z[q] = 0.0f;
        float acc = 0.0f;
        if constexpr (FPO_LDG256 && fused_ldg256(N1, N2)) {
            // 32-byte loads: both record strides are multiples of 8 floats
#pragma unroll
            for (int q = 0; q < (N1 + 7) / 8; ++q) {
                float wv[8];
                ldg256(reinterpret_cast<const float *>(sr) + 8 * q, wv);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (8 * q + j < N1) acc = fmaf(wv[j], bsrc[(8 * q + j) * bstride], acc);
            }
#pragma unroll
            for (int q = 0; q < (27 * N2 + 7) / 8; ++q) {
                float wv[8];
                ldg256(zr + 8 * q, wv);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int e = 8 * q + j;
                    if (e < 27 * N2) z[e / N2] = fmaf(wv[j], bz[e % N2], z[e / N2]);
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < (N1 + 3) / 4; ++q) {
                const float4 w = __ldg(sr + q);
                const float wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (4 * q + j < N1) acc = fmaf(wv[j], bsrc[(4 * q + j) * bstride], acc);
            }
#pragma unroll
            for (int q4 = 0; q4 < (27 * N2 + 3) / 4; ++q4) {
                const float4 w = __ldg(reinterpret_cast<const float4 *>(zr) + q4);
                const float wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int e = 4 * q4 + j;
                    if (e < 27 * N2) z[e / N2] = fmaf(wv[j], bz[e % N2], z[e / N2]);
                }
            }
        }
        sigma = fmaxf(acc, 0.0f);
    }
    float col[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float sacc = 0.0f;
#pragma unroll
        for (int k = 0; k < 9; ++k) sacc = fmaf(z[9 * c + k], R.Y[k], sacc);
        col[c] = sigmoidf_(sacc);
    }
    const float e = __expf(-sigma * delta);
    const float w = R.T * (1.0f - e);
    R.C0 = fmaf(w, col[0], R.C0);
    R.C1 = fmaf(w, col[1], R.C1);
    R.C2 = fmaf(w, col[2], R.C2);
    R.T *= e;
    if (DBG) {
        if (p.flags & FPO_FLAG_RECORD_VISITS) {
            if (R.n_visits < p.visit_cap)
                p.visit_log[(size_t)R.ray * p.visit_cap + R.n_visits] = p.perm[leaf];
            else
                atomicOr(p.status, STATUS_VISIT_OVERFLOW);
        }
        if (p.flags & FPO_FLAG_MARK_LEAVES) p.leaf_mark[p.perm[leaf]] = 1;
    }
    ++R.n_visits;
    return R.T < p.stop_T;
}

__device__ __forceinline__ bool step_cap(const TraverseParams &p, RayState &R)
{
    if (++R.steps > p.max_steps) {
        atomicOr(p.status, STATUS_TRAVERSAL_LIMIT);
        return true;
    }
    return false;
}

// Fused mode: the coefficient records of the next leaf (672 B at n1 = 31,
// n2 = 5) are pulled into L2 by two bulk prefetches while the current leaf is
// shaded, so its 32-byte loads hit L2 instead of HBM.
__device__ __forceinline__ void prefetch_records(const TraverseParams &p, uint32_t leaf, int n1, int n2)
{
    const float4 *sr = p.sig + (size_t)leaf * p.sig_stride4;
    const float *zr = p.zc + (size_t)leaf * p.z_stride;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(sr), "r"((uint32_t)(p.sig_stride4 * 16)));
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(zr), "r"((uint32_t)(p.z_stride * 4)));
    (void)n1;
    (void)n2;
}

// One step of the software-pipelined walk: the exit of cube `cb` (which
// holds R.P), the next cube located and its table record (or coefficient
// records) prefetched before `cb` is shaded, so the record's latency hides
// behind the shading arithmetic; then the move.  `cb` becomes the next cube.
// Returns false once the ray is finished (left the grid, early stop, or
// step cap).
template <int TM, bool DBG, int N1, int N2>
__device__ __forceinline__ bool pipelined_step(const TraverseParams &p, const float *bsrc, int bstride,
                                               const uint32_t *__restrict__ s_nodes, uint32_t *s_stack,
                                               int stride, RayState &R, Cube &cb)
{
    const int D = p.depth, G = 1 << D;
    int m, lo[3], csz;
    const float tx = cube_exit(R, D, cb.lvl, m, lo, csz);
    int Pn[3];
    const bool inside = next_cell(R, G, m, lo, csz, tx, Pn);
    Cube nx;
    nx.kind = ROOT_EMPTY;
    if (FPO_PREFETCH && inside) {
        const uint32_t diff = (uint32_t)((R.P[0] ^ Pn[0]) | (R.P[1] ^ Pn[1]) | (R.P[2] ^ Pn[2]));
        nx = locate(p, s_nodes, s_stack, stride, Pn, D - 1 - (31 - __clz(diff)));
        if (nx.kind == ROOT_LEAF) {
            if constexpr (TM == TM_TABLE_F32) {
                asm volatile("prefetch.global.L1 [%0];" ::"l"(table_record(p, nx.leaf)));
                if (FPO_PREFETCH_SIBLINGS)  // the aligned group of 4 lines holding it (siblings are adjacent)
                    asm volatile("cp.async.bulk.prefetch.L2.global [%0], 512;" ::"l"(table_record(p, nx.leaf & ~3u)));
            } else if constexpr (TM == TM_TABLE_F16) {
                asm volatile("prefetch.global.L1 [%0];" ::"l"(table_record_f16(p, nx.leaf)));
                if (FPO_PREFETCH_SIBLINGS)
                    asm volatile("cp.async.bulk.prefetch.L2.global [%0], 512;" ::"l"(table_record_f16(p, nx.leaf & ~7u)));
            } else {
                prefetch_records(p, nx.leaf, N1, N2);
            }
        }
    }
    if (cb.kind == ROOT_LEAF && tx > R.t)
        if (shade<TM, DBG, N1, N2>(p, bsrc, bstride, R, cb.leaf, tx - R.t)) return false;
    if (!inside) return false;
    move_to(R, D, Pn, tx);
    if (step_cap(p, R)) return false;
    if (FPO_PREFETCH)
        cb = nx;
    else
        cb = locate(p, s_nodes, s_stack, stride, R.P, R.lvl_start);
    return true;
}

// A whole ray (lane-loop schedule).
template <int TM, bool DBG, int N1, int N2>
__device__ void trace_ray(const TraverseParams &p, const float *bsrc, int bstride,
                          const uint32_t *__restrict__ s_nodes, uint32_t *s_stack, int stride,
                          RayState &R)
{
    Cube cb = locate(p, s_nodes, s_stack, stride, R.P, R.lvl_start);
    while (pipelined_step<TM, DBG, N1, N2>(p, bsrc, bstride, s_nodes, s_stack, stride, R, cb)) {
    }
}

}  // namespace

namespace {

// CTA prologue: stage the top n_smem_nodes nodes in shared memory; the frame
// basis (Eq. 8 at the shared t, FP64 then FP32) and the camera frame (FP64).
__device__ void frame_prologue(const TraverseParams &p, uint32_t *s_nodes, FrameShared &fs)
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

// Ray k (0..31) of a tile: a camera pixel of a TILE_W x TILE_H block, or an
// explicit ray.
__device__ __forceinline__ bool tile_ray(const TraverseParams &p, uint32_t tile, uint32_t k, uint32_t &ray,
                                         int &px, int &py)
{
    if (p.fr.mode == FPO_RAYS_CAMERA) {
        // row-major tiles: the tiles in flight form one band of rows, whose
        // table lines stay in L2
        const uint32_t tx = tile % p.tiles_x, ty = tile / p.tiles_x;
        px = (int)(tx * TILE_W + k % TILE_W);
        py = (int)(ty * TILE_H + k / TILE_W);
        ray = (uint32_t)py * p.fr.width + (uint32_t)px;
        return px < (int)p.fr.width && py < (int)p.fr.height;
    }
    ray = tile * 32 + k;
    return ray < p.fr.n_rays;
}

}  // namespace

// Persistent kernel: a grid of (SM count x resident CTAs) whose warps pull
// warp-sized tiles (TILE_W x TILE_H pixels, or 32 consecutive explicit rays) from one
// atomic counter.  Warp-level ray compaction: every lane holds its own ray;
// when at least REFILL_MIN lanes are idle, the warp hands them the next rays
// of its current tile (fetching a new tile when that one is used up), so
// long rays do not leave most of a warp idle.  Each CTA first stages the top
// n_smem_nodes nodes of the breadth-first node array and the frame constants
// in shared memory.  The last CTA to finish resets the counter.
// Register caps: 64 lets four 256-thread CTAs share an SM in materialised
// mode (measured fastest of 48..80 on the 3.5M-leaf body at 1080p); the fused
// per-visit IDFT needs more.
#ifndef FPO_TRAV_MAXNREG_MAT
#define FPO_TRAV_MAXNREG_MAT 64
#endif
#ifndef FPO_TRAV_MAXNREG_FUSED
#define FPO_TRAV_MAXNREG_FUSED 128
#endif

template <int TM, bool DBG, int N1, int N2, bool COMPACT>
__global__ void __maxnreg__(TM ? FPO_TRAV_MAXNREG_MAT : FPO_TRAV_MAXNREG_FUSED) traverse_kernel(const __grid_constant__ TraverseParams p)
{
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ FrameShared fs;
    const int stride = blockDim.x;
    uint32_t *s_nodes = smem;
    uint32_t *s_stack = smem + p.n_smem_nodes * 8;
    float *s_bray = reinterpret_cast<float *>(s_stack + STACK_LEVELS * stride);
    const bool prt = TM == TM_FUSED && p.fr.mode == FPO_RAYS_EXPLICIT && p.fr.rt != nullptr;

    frame_prologue(p, s_nodes, fs);
    __syncthreads();

    const int lane = threadIdx.x & 31;
    uint32_t *my_stack = s_stack + threadIdx.x;
    float *my_b = s_bray + threadIdx.x;
    const float *bsrc = prt ? my_b : fs.b;
    const int bstride = prt ? stride : 1;

    auto grab_tile = [&]() -> uint32_t {
        uint32_t tl = 0;
        if (lane == 0) tl = atomicAdd(p.tiles, 1u);
        return __shfl_sync(0xffffffffu, tl, 0);
    };
    auto finish = [&](const RayState &R) {
        write_result(p, R, DBG);
        if (DBG && (p.flags & FPO_FLAG_STATS)) {
            atomicAdd(p.stats, (unsigned long long)R.steps + 1ull);
            atomicAdd(p.stats + 1, (unsigned long long)R.n_visits);
            atomicAdd(p.stats + 2, 1ull);
        }
    };

    if constexpr (!COMPACT) {
        // One tile per warp at a time; every lane runs its ray to the end.
        for (;;) {
            const uint32_t tile = grab_tile();
            if (tile >= p.n_tiles) break;
            uint32_t ray;
            int px = 0, py = 0;
            if (tile_ray(p, tile, (uint32_t)lane, ray, px, py)) {
                RayState R;
                if (init_ray<DBG>(p, fs, prt, my_b, stride, my_stack, R, ray, px, py)) {
                    trace_ray<TM, DBG, N1, N2>(p, bsrc, bstride, s_nodes, my_stack, stride, R);
                    finish(R);
                }
            }
        }
    } else {
        // Warp-level ray compaction: once refill_min lanes are idle, they take
        // the next rays of the warp's current tile (a new tile when it is used
        // up); lanes take up to inner_steps steps between two checks.
        const uint32_t lt_mask = (1u << lane) - 1u;
        const uint32_t refill_min = p.refill_min;
        uint32_t cur_tile = grab_tile();  // warp-uniform cursor: tile and next ray in it
        uint32_t cur_next = 0;
        RayState R;
        Cube cb;  // the cube holding R.P, located ahead (pipelined step)
        cb.kind = ROOT_EMPTY;
        cb.leaf = 0;
        cb.lvl = 0;
        bool active = false;
        for (;;) {
            uint32_t idle = __ballot_sync(0xffffffffu, !active);
            if ((uint32_t)__popc(idle) >= refill_min) {
                while (idle && cur_tile < p.n_tiles) {
                    const uint32_t take = min(32u - cur_next, (uint32_t)__popc(idle));
                    const uint32_t rank = __popc(idle & lt_mask);
                    if (((idle >> lane) & 1u) && rank < take) {
                        uint32_t ray;
                        int px = 0, py = 0;
                        if (tile_ray(p, cur_tile, cur_next + rank, ray, px, py)) {
                            active = init_ray<DBG>(p, fs, prt, my_b, stride, my_stack, R, ray, px, py);
                            if (active) cb = locate(p, s_nodes, my_stack, stride, R.P, R.lvl_start);
                        }
                    }
                    cur_next += take;
                    if (cur_next >= 32) {
                        cur_tile = grab_tile();
                        cur_next = 0;
                    }
                    idle = __ballot_sync(0xffffffffu, !active);
                    if ((uint32_t)__popc(idle) < refill_min) break;
                }
            }
            if (!__any_sync(0xffffffffu, active)) break;
            if (active) {
#pragma unroll 1
                for (uint32_t k = 0; k < p.inner_steps; ++k) {
                    if (!pipelined_step<TM, DBG, N1, N2>(p, bsrc, bstride, s_nodes, my_stack, stride, R, cb)) {
                        finish(R);
                        active = false;
                        break;
                    }
                }
            }
        }
    }
    // The last warp of the grid to finish resets the tile counter for the
    // next launch (every warp has made its final grab before counting itself).
    if (lane == 0) {
        __threadfence();
        const uint32_t done = atomicAdd(p.tiles + 1, 1u);
        if (done == gridDim.x * (blockDim.x / 32) - 1) {
            atomicExch(p.tiles, 0u);
            atomicExch(p.tiles + 1, 0u);
        }
    }
}


int traverse_smem_bytes(uint32_t n_smem_nodes, bool per_ray_basis, int threads)
{
    return (int)(n_smem_nodes * 32u + STACK_LEVELS * threads * 4u +
                 (per_ray_basis ? 32u * threads * 4u : 0u));
}


template <int TM, bool DBG, int N1, int N2, bool COMPACT>
static int launch_t(const TraverseParams &p, int sm_count, cudaStream_t s)
{
    const bool prt = TM == TM_FUSED && p.fr.mode == FPO_RAYS_EXPLICIT && p.fr.rt != nullptr;
    const int threads = p.block_threads;
    const int smem = traverse_smem_bytes(p.n_smem_nodes, prt, threads);
    auto k = traverse_kernel<TM, DBG, N1, N2, COMPACT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 p.carveout > 0 ? p.carveout : (int)cudaSharedmemCarveoutDefault);
    if (e != cudaSuccess) return (int)e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem);
    if (e != cudaSuccess) return (int)e;
    if (per_sm < 1) per_sm = 1;
    if (p.max_ctas_per_sm > 0 && per_sm > p.max_ctas_per_sm) per_sm = p.max_ctas_per_sm;
    uint64_t blocks = (uint64_t)sm_count * per_sm;
    const uint64_t need = (p.n_tiles + (threads / 32) - 1) / (threads / 32);
    if (need < blocks) blocks = need ? need : 1;
    k<<<(unsigned)blocks, threads, smem, s>>>(p);
    return (int)cudaGetLastError();
}

// The compaction schedule (refill_min < 32) or the plain one, each with or
// without the debug outputs (visit logs, final T, leaf marks, counters).
template <int TM, int N1, int N2>
static int launch_sched(const TraverseParams &p, bool debug, int sm_count, cudaStream_t s)
{
    if (p.refill_min < 32)
        return debug ? launch_t<TM, true, N1, N2, true>(p, sm_count, s) : launch_t<TM, false, N1, N2, true>(p, sm_count, s);
    return debug ? launch_t<TM, true, N1, N2, false>(p, sm_count, s) : launch_t<TM, false, N1, N2, false>(p, sm_count, s);
}

static int launch_fused(const TraverseParams &p, bool debug, int sm_count, cudaStream_t s)
{
    // Fused per-visit IDFT: compile-time Fourier sizes (the settings of Tab. 3).
    if (p.n1 == 31 && p.n2 == 5) return launch_sched<TM_FUSED, 31, 5>(p, debug, sm_count, s);
    if (p.n1 == 11 && p.n2 == 5) return launch_sched<TM_FUSED, 11, 5>(p, debug, sm_count, s);
    if (p.n1 == 21 && p.n2 == 5) return launch_sched<TM_FUSED, 21, 5>(p, debug, sm_count, s);
    if (p.n1 == 31 && p.n2 == 11) return launch_sched<TM_FUSED, 31, 11>(p, debug, sm_count, s);
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
        return p.half_table ? launch_sched<TM_TABLE_F16, 0, 0>(p, debug, sm_count, s)
                            : launch_sched<TM_TABLE_F32, 0, 0>(p, debug, sm_count, s);
    return launch_fused(p, debug, sm_count, s);
}


// ---------------------------------------------------------------------------
// Adjoint of the render (Sec. 4.3: back-propagation through the IDFT).
//
// Each ray is replayed front to back with the fused per-visit IDFT (the same
// stepping and arithmetic as the fused forward, so the same segments and the
// same early stop), recomputing the transmittance instead of storing
// samples.  With w_j = T_j alpha_j and C the forward colour (which includes
// T_end bg), S_j = C - sum_{k<=j} w_k c_k is the colour behind segment j and
//   dL/dsigma_j = delta_j sum_c g_c (T_{j+1} c_jc - S_jc),
//   dL/du_jc    = g_c w_j c_jc (1 - c_jc),   u = sum_k z_ck Y_k,
//   dL/dk_sigma_i += dL/dsigma_j [sigma_raw > 0] IDFT_i(t),
//   dL/dk_cki     += dL/du_jc Y_k IDFT_i(t),
// accumulated with 16-byte vector atomics (one 8-byte atomic at an unaligned
// end) into the canonical gradient row of the leaf's upload id.

template <int N1, int N2>
__device__ void backward_ray(const BackwardParams &q, const float *bsrc, int bstride,
                             const uint32_t *__restrict__ s_nodes, uint32_t *s_stack, int stride,
                             RayState &R)
{
    constexpr int NC = N1 + 27 * N2;
    static_assert(NC % 2 == 0, "gradient rows are written in pairs");
    const TraverseParams &p = q.tp;
    const int D = p.depth, G = 1 << D;
    const float g0 = q.dL_drgb[3 * (size_t)R.ray], g1 = q.dL_drgb[3 * (size_t)R.ray + 1],
                g2 = q.dL_drgb[3 * (size_t)R.ray + 2];
    const float Cf0 = q.out_rgb[3 * (size_t)R.ray], Cf1 = q.out_rgb[3 * (size_t)R.ray + 1],
                Cf2 = q.out_rgb[3 * (size_t)R.ray + 2];
    float P0 = 0.0f, P1 = 0.0f, P2 = 0.0f;  // sum_{k<=j} w_k c_k
    float bz[N2];  // the density basis stays in shared memory (bsrc)
#pragma unroll
    for (int i = 0; i < N2; ++i) bz[i] = bsrc[i * bstride];
    Cube cb = locate(p, s_nodes, s_stack, stride, R.P, R.lvl_start);
    for (;;) {
        int m, lo[3], csz;
        const float tx = cube_exit(R, D, cb.lvl, m, lo, csz);
        // as in the forward: locate the next cube and prefetch its records
        // before this one is processed
        int Pn[3];
        const bool inside = next_cell(R, G, m, lo, csz, tx, Pn);
        Cube nx;
        nx.kind = ROOT_EMPTY;
        if (FPO_PREFETCH && inside) {
            const uint32_t diff = (uint32_t)((R.P[0] ^ Pn[0]) | (R.P[1] ^ Pn[1]) | (R.P[2] ^ Pn[2]));
            nx = locate(p, s_nodes, s_stack, stride, Pn, D - 1 - (31 - __clz(diff)));
            if (nx.kind == ROOT_LEAF) prefetch_records(p, nx.leaf, N1, N2);
        }
        if (cb.kind == ROOT_LEAF && tx > R.t) {
            const float delta = tx - R.t;
            const float *sr = reinterpret_cast<const float *>(p.sig + (size_t)cb.leaf * p.sig_stride4);
            const float *zr = p.zc + (size_t)cb.leaf * p.z_stride;
            constexpr int VW = (FPO_LDG256 && fused_ldg256(N1, N2)) ? 8 : 4;  // floats per load
            float sraw = 0.0f;
#pragma unroll
            for (int k4 = 0; k4 < (N1 + VW - 1) / VW; ++k4) {
                float wv[VW];
                load_vec<VW>(sr + VW * k4, wv);
#pragma unroll
                for (int j = 0; j < VW; ++j)
                    if (VW * k4 + j < N1) sraw = fmaf(wv[j], bsrc[(VW * k4 + j) * bstride], sraw);
            }
            const float sigma = fmaxf(sraw, 0.0f);
            float z[27];
#pragma unroll
            for (int k = 0; k < 27; ++k) z[k] = 0.0f;
#pragma unroll
            for (int k4 = 0; k4 < (27 * N2 + VW - 1) / VW; ++k4) {
                float wv[VW];
                load_vec<VW>(zr + VW * k4, wv);
#pragma unroll
                for (int j = 0; j < VW; ++j) {
                    const int e = VW * k4 + j;
                    if (e < 27 * N2) z[e / N2] = fmaf(wv[j], bz[e % N2], z[e / N2]);
                }
            }
            float col[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float u = 0.0f;
#pragma unroll
                for (int k = 0; k < 9; ++k) u = fmaf(z[9 * c + k], R.Y[k], u);
                col[c] = sigmoidf_(u);
            }
            const float e = __expf(-sigma * delta);
            const float w = R.T * (1.0f - e);
            const float Tn = R.T * e;
            P0 = fmaf(w, col[0], P0);
            P1 = fmaf(w, col[1], P1);
            P2 = fmaf(w, col[2], P2);
            const float gs = delta * (g0 * (Tn * col[0] - (Cf0 - P0)) + g1 * (Tn * col[1] - (Cf1 - P1)) +
                                      g2 * (Tn * col[2] - (Cf2 - P2)));
            const float dsr = sraw > 0.0f ? gs : 0.0f;
            const float gu[3] = {g0 * w * col[0] * (1.0f - col[0]), g1 * w * col[1] * (1.0f - col[1]),
                                 g2 * w * col[2] * (1.0f - col[2])};
            const uint32_t id = p.perm[cb.leaf];
            float *row = q.dL_dcoeffs + (size_t)id * NC;
            if (q.leaf_mark) q.leaf_mark[id] = 1;
            // dL/dk for element el of the row (compile-time el)
            auto gval = [&](int el) -> float {
                if (el < N1) return dsr * bsrc[el * bstride];
                const int j = el - N1, c = j / (9 * N2), k = (j / N2) % 9, i = j % N2;
                return gu[c] * R.Y[k] * bz[i];
            };
            // 16-byte vector atomics; a row that starts 8 bytes past a 16-byte
            // boundary (NC = 2 mod 4, odd id) opens with one 8-byte atomic
            if (NC % 4 == 0 || (id & 1u) == 0u) {
#pragma unroll
                for (int e4 = 0; e4 < NC / 4; ++e4)
                    atomicAdd(reinterpret_cast<float4 *>(row) + e4,
                              make_float4(gval(4 * e4), gval(4 * e4 + 1), gval(4 * e4 + 2), gval(4 * e4 + 3)));
                if constexpr (NC % 4 == 2)
                    atomicAdd(reinterpret_cast<float2 *>(row + NC - 2), make_float2(gval(NC - 2), gval(NC - 1)));
            } else {
                atomicAdd(reinterpret_cast<float2 *>(row), make_float2(gval(0), gval(1)));
#pragma unroll
                for (int e4 = 0; e4 < NC / 4; ++e4)
                    atomicAdd(reinterpret_cast<float4 *>(row + 2) + e4,
                              make_float4(gval(2 + 4 * e4), gval(3 + 4 * e4), gval(4 + 4 * e4), gval(5 + 4 * e4)));
            }
            R.T = Tn;
            if (R.T < p.stop_T) return;
        }
        if (!inside) return;
        move_to(R, D, Pn, tx);
        if (step_cap(p, R)) return;
        if (FPO_PREFETCH)
            cb = nx;
        else
            cb = locate(p, s_nodes, s_stack, stride, R.P, R.lvl_start);
    }
}

template <int N1, int N2>
__global__ void __maxnreg__(128) backward_kernel(const __grid_constant__ BackwardParams q)
{
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ FrameShared fs;
    const TraverseParams &p = q.tp;
    const int stride = blockDim.x;
    uint32_t *s_nodes = smem;
    uint32_t *s_stack = smem + p.n_smem_nodes * 8;
    float *s_bray = reinterpret_cast<float *>(s_stack + STACK_LEVELS * stride);
    const bool prt = p.fr.mode == FPO_RAYS_EXPLICIT && p.fr.rt != nullptr;
    frame_prologue(p, s_nodes, fs);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    uint32_t *my_stack = s_stack + threadIdx.x;
    float *my_b = s_bray + threadIdx.x;
    const float *bsrc = prt ? my_b : fs.b;
    const int bstride = prt ? stride : 1;
    for (;;) {
        uint32_t tile = 0;
        if (lane == 0) tile = atomicAdd(p.tiles, 1u);
        tile = __shfl_sync(0xffffffffu, tile, 0);
        if (tile >= p.n_tiles) break;
        uint32_t ray;
        int px = 0, py = 0;
        if (!tile_ray(p, tile, (uint32_t)lane, ray, px, py)) continue;
        RayState R;
        if (!init_ray_geom(p, fs, prt, my_b, stride, my_stack, R, ray, px, py)) continue;
        backward_ray<N1, N2>(q, bsrc, bstride, s_nodes, my_stack, stride, R);
    }
    if (lane == 0) {
        __threadfence();
        const uint32_t done = atomicAdd(p.tiles + 1, 1u);
        if (done == gridDim.x * (blockDim.x / 32) - 1) {
            atomicExch(p.tiles, 0u);
            atomicExch(p.tiles + 1, 0u);
        }
    }
}

template <int N1, int N2>
static int launch_b(const BackwardParams &q, int sm_count, cudaStream_t s)
{
    const TraverseParams &p = q.tp;
    const bool prt = p.fr.mode == FPO_RAYS_EXPLICIT && p.fr.rt != nullptr;
    const int threads = 256;
    const int smem = traverse_smem_bytes(p.n_smem_nodes, prt, threads);
    auto k = backward_kernel<N1, N2>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 p.carveout > 0 ? p.carveout : (int)cudaSharedmemCarveoutDefault);
    if (e != cudaSuccess) return (int)e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem);
    if (e != cudaSuccess) return (int)e;
    if (per_sm < 1) per_sm = 1;
    if (p.max_ctas_per_sm > 0 && per_sm > p.max_ctas_per_sm) per_sm = p.max_ctas_per_sm;
    uint64_t blocks = (uint64_t)sm_count * per_sm;
    const uint64_t need = (p.n_tiles + (threads / 32) - 1) / (threads / 32);
    if (need < blocks) blocks = need ? need : 1;
    k<<<(unsigned)blocks, threads, smem, s>>>(q);
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Gradient-check replay (FPO_FLAG_FP64_GRADCHECK).  The FP32 stepping above
// decides which leaves the ray visits and in which order (as the forward
// does); each visited leaf's segment is re-measured by an FP64 slab test of
// its box along the FP64-normalised ray, and the IDFT (Eq. 7, 9), the SH
// colour (Eq. 1), the transmittance products and S_j are FP64.  Two replays
// per ray: the first composites the FP64 colour C (with T_end bg), the second
// forms S_j = C - sum_{k<=j} w_k c_k and the gradients, accumulated with FP64
// atomics.

struct Ray64 {
    double go[3], gd[3];  // origin and unit direction, in grid units
    double Y[9];          // real SH of the unit direction
    double b[MAX_BASIS];  // Eq. 8 at the ray's time
};

__device__ __forceinline__ void sh_basis64(double x, double y, double z, double Y[9])
{
    const double c0 = 0.28209479177387814, c1 = 0.48860251190291992, c2 = 1.09254843059207907,
                 c3 = 0.31539156525252005, c4 = 0.54627421529603959;
    Y[0] = c0;
    Y[1] = -c1 * y;
    Y[2] = c1 * z;
    Y[3] = -c1 * x;
    Y[4] = c2 * x * y;
    Y[5] = -c2 * y * z;
    Y[6] = c3 * (3.0 * z * z - 1.0);
    Y[7] = -c2 * x * z;
    Y[8] = c4 * (x * x - y * y);
}

// The FP64 ray of ray index `ray` (camera pixel or explicit ray), as the
// oracle forms it: camera frame and pixel direction in FP64, or the FP32
// inputs widened, then normalised in FP64.
__device__ void ray64_setup(const TraverseParams &p, uint32_t ray, int px, int py, Ray64 &r)
{
    double o[3], d[3], t = p.fr.t;
    if (p.fr.mode == FPO_RAYS_CAMERA) {
        double f[3], rt[3], u[3];
        for (int k = 0; k < 3; ++k) f[k] = p.fr.target[k] - p.fr.eye[k];
        const double fl = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
        for (int k = 0; k < 3; ++k) f[k] /= fl;
        rt[0] = f[1] * p.fr.up[2] - f[2] * p.fr.up[1];
        rt[1] = f[2] * p.fr.up[0] - f[0] * p.fr.up[2];
        rt[2] = f[0] * p.fr.up[1] - f[1] * p.fr.up[0];
        const double rl = sqrt(rt[0] * rt[0] + rt[1] * rt[1] + rt[2] * rt[2]);
        for (int k = 0; k < 3; ++k) rt[k] /= rl;
        u[0] = rt[1] * f[2] - rt[2] * f[1];
        u[1] = rt[2] * f[0] - rt[0] * f[2];
        u[2] = rt[0] * f[1] - rt[1] * f[0];
        const double th = tan(0.5 * p.fr.fov_y_deg * 3.14159265358979323846 / 180.0);
        const double sx = (2.0 * ((double)px + 0.5) / (double)p.fr.width - 1.0) * th * ((double)p.fr.width / (double)p.fr.height);
        const double sy = (1.0 - 2.0 * ((double)py + 0.5) / (double)p.fr.height) * th;
        for (int k = 0; k < 3; ++k) {
            o[k] = p.fr.eye[k];
            d[k] = f[k] + sx * rt[k] + sy * u[k];
        }
    } else {
        for (int k = 0; k < 3; ++k) {
            o[k] = (double)p.fr.ro[3 * (size_t)ray + k];
            d[k] = (double)p.fr.rd[3 * (size_t)ray + k];
        }
        if (p.fr.rt) t = (double)p.fr.rt[ray];
    }
    const double dl = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int k = 0; k < 3; ++k) {
        d[k] /= dl;
        r.go[k] = (o[k] - p.amin64[k]) * p.grid_scale64;
        r.gd[k] = d[k] * p.grid_scale64;
    }
    sh_basis64(d[0], d[1], d[2], r.Y);
    const int nb = p.n1 > p.n2 ? p.n1 : p.n2;
    const double u = t / p.fr.period_T;
    for (int i = 0; i < nb; ++i) r.b[i] = (i & 1) ? sinpi((double)(i + 1) * u) : cospi((double)i * u);
}

// Length (along the unit ray, t >= 0) of the ray inside the box
// [lo, lo + csz]^3 (grid units): the FP64 slab test.
__device__ __forceinline__ double segment64(const Ray64 &r, const int lo[3], int csz)
{
    double t0 = 0.0, t1 = 1.0e300;
    for (int a = 0; a < 3; ++a) {
        if (r.gd[a] == 0.0) continue;
        const double ta = ((double)lo[a] - r.go[a]) / r.gd[a], tb = ((double)(lo[a] + csz) - r.go[a]) / r.gd[a];
        t0 = fmax(t0, fmin(ta, tb));
        t1 = fmin(t1, fmax(ta, tb));
    }
    return t1 - t0;
}

// One replay of a ray: pass 0 composites C (returned with T_end bg added);
// pass 1 accumulates the gradients with C from pass 0.
template <int N1, int N2>
__device__ void replay_fp64(const BackwardParams &q, RayState R, const Ray64 &r, int pass, double C[3],
                            const uint32_t *__restrict__ s_nodes, uint32_t *s_stack, int stride)
{
    constexpr int NC = N1 + 27 * N2;
    const TraverseParams &p = q.tp;
    const int D = p.depth, G = 1 << D;
    double g[3] = {0.0, 0.0, 0.0};
    if (pass == 1)
        for (int c = 0; c < 3; ++c) g[c] = (double)q.dL_drgb[3 * (size_t)R.ray + c];
    double T = 1.0, P[3] = {0.0, 0.0, 0.0};
    for (;;) {
        const Cube cb = locate(p, s_nodes, s_stack, stride, R.P, R.lvl_start);
        int m, lo[3], csz;
        const float tx = cube_exit(R, D, cb.lvl, m, lo, csz);
        if (cb.kind == ROOT_LEAF && tx > R.t) {
            const double delta = segment64(r, lo, csz);
            const float *sr = reinterpret_cast<const float *>(p.sig + (size_t)cb.leaf * p.sig_stride4);
            const float *zr = p.zc + (size_t)cb.leaf * p.z_stride;
            double sraw = 0.0;
            for (int i = 0; i < N1; ++i) sraw += (double)sr[i] * r.b[i];
            const double sigma = sraw > 0.0 ? sraw : 0.0;
            double col[3];
            for (int c = 0; c < 3; ++c) {
                double u = 0.0;
                for (int k = 0; k < 9; ++k) {
                    double z = 0.0;
                    for (int i = 0; i < N2; ++i) z += (double)zr[(c * 9 + k) * N2 + i] * r.b[i];
                    u += z * r.Y[k];
                }
                col[c] = 1.0 / (1.0 + exp(-u));
            }
            const double e = exp(-sigma * delta);
            const double w = T * (1.0 - e), Tn = T * e;
            for (int c = 0; c < 3; ++c) P[c] += w * col[c];
            if (pass == 1) {
                double gs = 0.0;
                for (int c = 0; c < 3; ++c) gs += g[c] * delta * (Tn * col[c] - (C[c] - P[c]));
                double *row = q.dL_dcoeffs64 + (size_t)p.perm[cb.leaf] * NC;
                if (sraw > 0.0)
                    for (int i = 0; i < N1; ++i) atomicAdd(row + i, gs * r.b[i]);
                for (int c = 0; c < 3; ++c) {
                    const double du = g[c] * w * col[c] * (1.0 - col[c]);
                    for (int k = 0; k < 9; ++k)
                        for (int i = 0; i < N2; ++i) atomicAdd(row + N1 + (c * 9 + k) * N2 + i, du * r.Y[k] * r.b[i]);
                }
                if (q.leaf_mark) q.leaf_mark[p.perm[cb.leaf]] = 1;
            }
            T = Tn;
            if (T < (double)p.stop_T) break;
        }
        int Pn[3];
        if (!next_cell(R, G, m, lo, csz, tx, Pn)) break;
        move_to(R, D, Pn, tx);
        if (step_cap(p, R)) break;
    }
    if (pass == 0)
        for (int c = 0; c < 3; ++c) C[c] = P[c] + T * (double)p.bg[c];
}

template <int N1, int N2>
__global__ void __launch_bounds__(128) backward_fp64_kernel(const __grid_constant__ BackwardParams q)
{
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ FrameShared fs;
    const TraverseParams &p = q.tp;
    const int stride = blockDim.x;
    uint32_t *s_nodes = smem;
    uint32_t *s_stack = smem + p.n_smem_nodes * 8;
    float *s_bray = reinterpret_cast<float *>(s_stack + STACK_LEVELS * stride);
    frame_prologue(p, s_nodes, fs);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    uint32_t *my_stack = s_stack + threadIdx.x;
    for (;;) {
        uint32_t tile = 0;
        if (lane == 0) tile = atomicAdd(p.tiles, 1u);
        tile = __shfl_sync(0xffffffffu, tile, 0);
        if (tile >= p.n_tiles) break;
        uint32_t ray;
        int px = 0, py = 0;
        if (!tile_ray(p, tile, (uint32_t)lane, ray, px, py)) continue;
        RayState R0;
        // the FP32 ray as the forward sets it up (it decides the stepping)
        if (!init_ray_geom(p, fs, false, s_bray + threadIdx.x, stride, my_stack, R0, ray, px, py)) continue;
        Ray64 r;
        ray64_setup(p, ray, px, py, r);
        double C[3];
        replay_fp64<N1, N2>(q, R0, r, 0, C, s_nodes, my_stack, stride);
        replay_fp64<N1, N2>(q, R0, r, 1, C, s_nodes, my_stack, stride);
    }
    if (lane == 0) {
        __threadfence();
        const uint32_t done = atomicAdd(p.tiles + 1, 1u);
        if (done == gridDim.x * (blockDim.x / 32) - 1) {
            atomicExch(p.tiles, 0u);
            atomicExch(p.tiles + 1, 0u);
        }
    }
}

template <int N1, int N2>
static int launch_b64(const BackwardParams &q, int sm_count, cudaStream_t s)
{
    const TraverseParams &p = q.tp;
    const int threads = 128;
    const int smem = traverse_smem_bytes(p.n_smem_nodes, false, threads);
    auto k = backward_fp64_kernel<N1, N2>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return (int)e;
    const uint64_t need = (p.n_tiles + (threads / 32) - 1) / (threads / 32);
    uint64_t blocks = (uint64_t)sm_count * 4;
    if (need < blocks) blocks = need ? need : 1;
    k<<<(unsigned)blocks, threads, smem, s>>>(q);
    return (int)cudaGetLastError();
}

int launch_backward(const BackwardParams &q, int sm_count, void *stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    const TraverseParams &p = q.tp;
    const bool fp64 = q.dL_dcoeffs64 != nullptr;
    if (p.n1 == 31 && p.n2 == 5) return fp64 ? launch_b64<31, 5>(q, sm_count, s) : launch_b<31, 5>(q, sm_count, s);
    if (p.n1 == 11 && p.n2 == 5) return fp64 ? launch_b64<11, 5>(q, sm_count, s) : launch_b<11, 5>(q, sm_count, s);
    if (p.n1 == 21 && p.n2 == 5) return fp64 ? launch_b64<21, 5>(q, sm_count, s) : launch_b<21, 5>(q, sm_count, s);
    if (p.n1 == 31 && p.n2 == 11) return fp64 ? launch_b64<31, 11>(q, sm_count, s) : launch_b<31, 11>(q, sm_count, s);
    return -1;
}

// ---------------------------------------------------------------------------
// Rows of `bytes` bytes (a multiple of 16) from upload order to internal
// leaf order: dst[i] = src[perm[i]].

__global__ void gather_rows_kernel(const uint4 *__restrict__ src, uint4 *__restrict__ dst,
                                   const uint32_t *__restrict__ perm, uint32_t n, uint32_t words)
{
    const uint64_t total = (uint64_t)n * words;
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t i = (uint32_t)(g / words), w = (uint32_t)(g % words);
        dst[g] = __ldg(src + (size_t)perm[i] * words + w);
    }
}

int launch_gather_rows(const void *src, void *dst, const uint32_t *perm, uint32_t n, uint32_t bytes,
                       int sm_count, void *stream)
{
    if (n == 0) return (int)cudaSuccess;
    const uint32_t words = bytes / 16;
    uint64_t blocks = ((uint64_t)n * words + 255) / 256;
    if (blocks > (uint64_t)sm_count * 32) blocks = (uint64_t)sm_count * 32;
    gather_rows_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(
        static_cast<const uint4 *>(src), static_cast<uint4 *>(dst), perm, n, words);
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Canonical coefficients (device, upload order) -> FP32 leaf records.
// One warp per leaf: lanes stride over the n1 + 27 n2 values (coalesced).

__global__ void __launch_bounds__(256) set_coeffs_kernel(const float *__restrict__ src, const uint32_t *__restrict__ perm,
                                                         float *sig, float *zc, uint32_t n_leaves, int n1, int n2,
                                                         int ss, int zs)
{
    const int lane = threadIdx.x & 31;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    const int nc = n1 + 27 * n2;
    for (uint32_t leaf = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; leaf < n_leaves; leaf += warps) {
        const float *row = src + (size_t)perm[leaf] * nc;
        for (int j = lane; j < nc; j += 32) {
            const float v = row[j];
            if (j < n1) sig[(size_t)leaf * ss + j] = v;
            else zc[(size_t)leaf * zs + (j - n1)] = v;
        }
    }
}

int launch_set_coeffs(const float *src, const uint32_t *perm, float *sig, float *zc, uint32_t n_leaves,
                      int n1, int n2, int sm_count, void *stream)
{
    if (n_leaves == 0) return (int)cudaSuccess;
    uint64_t blocks = ((uint64_t)n_leaves * 32 + 255) / 256;
    if (blocks > (uint64_t)sm_count * 16) blocks = (uint64_t)sm_count * 16;
    set_coeffs_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(src, perm, sig, zc, n_leaves, n1, n2,
                                                                           sig_stride(n1), z_stride(n2));
    return (int)cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Per-leaf DFT (Sec. 4.2, Eq. 10-12): coefficients from the values a leaf
// takes at frames t = 1..T (the unified per-frame octrees).  One thread per
// output coefficient (leaf, j): coalesced stores; the threads of one series
// read the same per-frame value (L1 broadcast).  The DFT weights
// (w_i / T) {cos, sin}, w_0 = 1, w_i = 2, come from FP64 into shared memory.

constexpr int DFT_MAX_T = 256;

__global__ void __launch_bounds__(256) dft_kernel(const float *__restrict__ values, float *__restrict__ coeffs,
                                                  uint32_t n_leaves, int n1, int n2, int T)
{
    __shared__ float s_w[32 * DFT_MAX_T];
    const int nb = n1 > n2 ? n1 : n2;
    for (int q = threadIdx.x; q < nb * T; q += blockDim.x) {
        const int i = q / T, t = q % T + 1;
        const double u = (double)t / (double)T;
        const double w = (i == 0 ? 1.0 : 2.0) / (double)T;
        s_w[q] = (float)(w * ((i & 1) ? sinpi((double)(i + 1) * u) : cospi((double)i * u)));
    }
    __syncthreads();
    const int nc = n1 + 27 * n2;
    const uint64_t total = (uint64_t)n_leaves * nc;
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t leaf = (uint32_t)(g / nc);
        const int j = (int)(g % nc);
        const int series = j < n1 ? 0 : 1 + (j - n1) / n2;
        const int i = j < n1 ? j : (j - n1) % n2;
        const float *x = values + (size_t)leaf * 28 + series;
        const float *w = s_w + i * T;
        float acc = 0.0f;
        for (int t = 0; t < T; ++t) acc = fmaf(__ldg(x + (size_t)t * n_leaves * 28), w[t], acc);
        coeffs[g] = acc;
    }
}

// Tiled version for n2 = 5 (the paper's size; any n1 <= 32): a CTA takes 32
// leaves at a time.  Frames arrive in chunks of DFT_TC, each chunk's 32 x 28
// values read with coalesced loads into shared memory; lane l of every warp
// owns leaf l: warp 0 accumulates the density series (n1 coefficients), warps
// 1..7 the 27 SH series (series w, w + 7, w + 14, w + 21; 5 coefficients
// each), with the weights of a frame read as float4 broadcasts.  The sums run
// over t in the same order as the kernel above, so both give the same bits.
// The 32 x nc outputs are staged in shared memory and written contiguously.
constexpr int DFT_TILE = 32, DFT_TC = 8, DFT_XPAD = 29, DFT_N2 = 5;

__global__ void __launch_bounds__(256) dft_tile_kernel(const float *__restrict__ values, float *__restrict__ coeffs,
                                                       uint32_t n_leaves, int n1, int T)
{
    extern __shared__ __align__(16) float dft_smem[];
    float *s_w = dft_smem;                          // [T][32]: weight of coefficient i at frame t
    float *s_x = s_w + (size_t)T * 32;              // [DFT_TC][32 leaves][DFT_XPAD]
    const int nc = n1 + 27 * DFT_N2;
    float *s_out = s_x + DFT_TC * DFT_TILE * DFT_XPAD;  // [32 leaves][nc]
    for (int q = threadIdx.x; q < 32 * T; q += blockDim.x) {
        const int t = q / 32, i = q % 32, nb = n1 > DFT_N2 ? n1 : DFT_N2;
        const double u = (double)(t + 1) / (double)T;
        const double w = (i == 0 ? 1.0 : 2.0) / (double)T;
        s_w[q] = i < nb ? (float)(w * ((i & 1) ? sinpi((double)(i + 1) * u) : cospi((double)i * u))) : 0.0f;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int ser[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) ser[q] = warp == 0 ? (q == 0 ? 0 : -1) : (warp + 7 * q <= 27 ? warp + 7 * q : -1);
    const uint32_t n_tiles = (n_leaves + DFT_TILE - 1) / DFT_TILE;
    for (uint32_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const uint32_t leaf0 = tile * DFT_TILE;
        const int nl = (int)min((uint32_t)DFT_TILE, n_leaves - leaf0);
        float acc[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) acc[i] = 0.0f;
        for (int t0 = 0; t0 < T; t0 += DFT_TC) {
            const int tc = min(DFT_TC, T - t0);
            __syncthreads();  // the previous chunk (and the weights) are done with
            if (tc == DFT_TC && nl == DFT_TILE && blockDim.x == 256) {
                // full chunk: 28 coalesced loads per thread, all in flight, then the stores
                constexpr int PER = DFT_TC * DFT_TILE * 28 / 256;
                float v[PER];
#pragma unroll
                for (int k = 0; k < PER; ++k) {
                    const int q = threadIdx.x + 256 * k, t = q / (DFT_TILE * 28), r = q % (DFT_TILE * 28);
                    v[k] = __ldg(values + ((size_t)(t0 + t) * n_leaves + leaf0) * 28 + r);
                }
#pragma unroll
                for (int k = 0; k < PER; ++k) {
                    const int q = threadIdx.x + 256 * k, t = q / (DFT_TILE * 28), r = q % (DFT_TILE * 28);
                    s_x[(t * DFT_TILE + r / 28) * DFT_XPAD + r % 28] = v[k];
                }
            } else {
                for (int q = threadIdx.x; q < tc * nl * 28; q += blockDim.x) {
                    const int t = q / (nl * 28), r = q % (nl * 28);
                    s_x[(t * DFT_TILE + r / 28) * DFT_XPAD + r % 28] =
                        __ldg(values + ((size_t)(t0 + t) * n_leaves + leaf0) * 28 + r);
                }
            }
            __syncthreads();
            if (lane < nl) {
                for (int t = 0; t < tc; ++t) {
                    const float *xr = s_x + (t * DFT_TILE + lane) * DFT_XPAD;
                    const float4 *wr = reinterpret_cast<const float4 *>(s_w + (size_t)(t0 + t) * 32);
                    if (warp == 0) {
                        const float x = xr[0];
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            const float4 w = wr[k];
                            acc[4 * k] = fmaf(x, w.x, acc[4 * k]);
                            acc[4 * k + 1] = fmaf(x, w.y, acc[4 * k + 1]);
                            acc[4 * k + 2] = fmaf(x, w.z, acc[4 * k + 2]);
                            acc[4 * k + 3] = fmaf(x, w.w, acc[4 * k + 3]);
                        }
                    } else {
                        const float4 w4 = wr[0];
                        const float w5 = s_w[(size_t)(t0 + t) * 32 + 4];
                        const float wv[DFT_N2] = {w4.x, w4.y, w4.z, w4.w, w5};
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            if (ser[q] < 0) continue;
                            const float x = xr[ser[q]];
#pragma unroll
                            for (int i = 0; i < DFT_N2; ++i) acc[q * DFT_N2 + i] = fmaf(x, wv[i], acc[q * DFT_N2 + i]);
                        }
                    }
                }
            }
        }
        if (lane < nl) {
            float *o = s_out + (size_t)lane * nc;
            if (warp == 0) {
#pragma unroll
                for (int i = 0; i < 32; ++i)
                    if (i < n1) o[i] = acc[i];
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (ser[q] < 0) continue;
#pragma unroll
                    for (int i = 0; i < DFT_N2; ++i) o[n1 + (ser[q] - 1) * DFT_N2 + i] = acc[q * DFT_N2 + i];
                }
            }
        }
        __syncthreads();
        for (int q = threadIdx.x; q < nl * nc; q += blockDim.x) coeffs[(size_t)leaf0 * nc + q] = s_out[q];
    }
}

// Bulk-copy version (the default), bit-equal to the two kernels above (each
// coefficient is summed over t in the same order).  Thread 0 moves each frame
// of a tile (32 leaves x 28 values: 3584 contiguous bytes) into a ring stage
// with one bulk asynchronous copy, completion counted in bytes on the stage's
// mbarrier, DFTB_STAGES units of DFTB_FPS frames ahead and across tile
// boundaries (a 16-byte cp.async version of this ring, with the tile
// kernel's eight warps, peaked at 1.14 ms on 512K leaves: the per-SM limit on
// outstanding requests).  Nine warps share a frame's work evenly: lane l owns
// leaf l; warps 0 and 1 the density coefficients 0..15 and 16..n1-1, warps
// 2..8 the 27 SH series (3 or 4 each, rotated by l / 8 so a warp's reads of
// one frame hit all 32 banks).  A wait that runs out (2 s;
// 1 ms for the first wait with FPO_FLAG_TEST_DEVICE_TIMEOUT) sets
// STATUS_DEVICE_TIMEOUT in *status (if given), writes NaN to every
// coefficient of the CTA's unfinished tiles, waits (bounded) for its copies
// in flight and returns.
// Measured on 512K leaves x 60 frames (frames per stage x stages): 12 x 2
// 0.79 ms, 8 x 2 0.87, 8 x 3 0.88, 10 x 2 0.85, 15 x 2 1.16, 20 x 2 1.10.
#ifndef FPO_DFT_BULK_FPS
#define FPO_DFT_BULK_FPS 12
#endif
#ifndef FPO_DFT_BULK_STAGES
#define FPO_DFT_BULK_STAGES 2
#endif
constexpr int DFTB_FPS = FPO_DFT_BULK_FPS, DFTB_STAGES = FPO_DFT_BULK_STAGES, DFTB_THREADS = 288;
constexpr int DFT_FRAME_FLOATS = DFT_TILE * 28;  // one frame of a tile

__global__ void __launch_bounds__(DFTB_THREADS) dft_bulk_kernel(const float *__restrict__ values,
                                                                float *__restrict__ coeffs, uint32_t n_leaves,
                                                                int n1, int T, uint32_t *status, bool test_timeout)
{
    extern __shared__ __align__(128) float dftb_smem[];
    __shared__ uint64_t bars[DFTB_STAGES];
    __shared__ uint64_t never;  // test_timeout: a barrier nothing signals
    __shared__ int s_fail;
    float *ring = dftb_smem;                                           // [stages][frames][32 leaves][28]
    float *s_w = ring + DFTB_STAGES * DFTB_FPS * DFT_FRAME_FLOATS;     // [T][32]
    const int nc = n1 + 27 * DFT_N2;
    float *s_out = s_w + (size_t)T * 32;                               // [32 leaves][nc]
    const uint32_t n_tiles = (n_leaves + DFT_TILE - 1) / DFT_TILE;
    const int groups = (T + DFTB_FPS - 1) / DFTB_FPS;
    const uint32_t my_tiles = blockIdx.x < n_tiles ? (n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const uint32_t units = my_tiles * (uint32_t)groups;
    auto unit_tile = [&](uint32_t u) { return blockIdx.x + (u / groups) * gridDim.x; };
    auto issue = [&](uint32_t u) {
        const uint32_t tile = unit_tile(u);
        const uint32_t leaf0 = tile * DFT_TILE;
        const uint32_t nl = min((uint32_t)DFT_TILE, n_leaves - leaf0);
        const int f0 = (int)(u % groups) * DFTB_FPS, nf = min(DFTB_FPS, T - f0);
        const int st = (int)(u % DFTB_STAGES);
        float *dst = ring + (size_t)st * DFTB_FPS * DFT_FRAME_FLOATS;
        ptx::mbar_arrive_expect_tx(&bars[st], (uint32_t)nf * nl * 112u);
        for (int f = 0; f < nf; ++f)
            ptx::bulk_g2s(dst + f * DFT_FRAME_FLOATS, values + ((size_t)(f0 + f) * n_leaves + leaf0) * 28, nl * 112u,
                          &bars[st]);
    };
    if (threadIdx.x == 0) {
        s_fail = 0;
        for (int st = 0; st < DFTB_STAGES; ++st) ptx::mbar_init(&bars[st], 1);
        ptx::mbar_init(&never, 1);
        ptx::fence_barrier_init();
        for (uint32_t u = 0; u < (uint32_t)DFTB_STAGES && u < units; ++u) issue(u);
    }
    for (int q = threadIdx.x; q < 32 * T; q += blockDim.x) {
        const int t = q / 32, i = q % 32, nb = n1 > DFT_N2 ? n1 : DFT_N2;
        const double u = (double)(t + 1) / (double)T;
        const double w = (i == 0 ? 1.0 : 2.0) / (double)T;
        s_w[q] = i < nb ? (float)(w * ((i & 1) ? sinpi((double)(i + 1) * u) : cospi((double)i * u))) : 0.0f;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool dens = warp < 2;
    const int d0 = 16 * warp;  // density warps: coefficients d0 .. d0 + 15
    int ser[4];                // SH warps: series, or -1
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int b = warp - 2 + 7 * q;
        ser[q] = !dens && b <= 26 ? 1 + (b + (lane >> 3)) % 27 : -1;
    }
    float acc[20];
#pragma unroll
    for (int i = 0; i < 20; ++i) acc[i] = 0.0f;
    uint32_t unit = 0;
    for (; unit < units; ++unit) {
        const int st = (int)(unit % DFTB_STAGES);
        const bool ok = test_timeout && unit == 0
                            ? ptx::mbar_wait_bounded(&never, 0, TEST_WAIT_LIMIT_NS)
                            : ptx::mbar_wait_bounded(&bars[st], (unit / DFTB_STAGES) & 1u, WAIT_LIMIT_NS);
        if (!ok) s_fail = 1;
        __syncthreads();
        if (s_fail) break;
        const uint32_t tile = unit_tile(unit);
        const uint32_t leaf0 = tile * DFT_TILE;
        const int nl = (int)min((uint32_t)DFT_TILE, n_leaves - leaf0);
        const int g = (int)(unit % groups), f0 = g * DFTB_FPS, nf = min(DFTB_FPS, T - f0);
        const float *stg = ring + (size_t)st * DFTB_FPS * DFT_FRAME_FLOATS;
        if (lane < nl && (!dens || d0 < n1)) {
            for (int f = 0; f < nf; ++f) {
                const float *xr = stg + f * DFT_FRAME_FLOATS + lane * 28;
                const float *wt = s_w + (size_t)(f0 + f) * 32;
                if (dens) {
                    const float x = xr[0];
                    const float4 *wr = reinterpret_cast<const float4 *>(wt + d0);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float4 w = wr[k];
                        acc[4 * k] = fmaf(x, w.x, acc[4 * k]);
                        acc[4 * k + 1] = fmaf(x, w.y, acc[4 * k + 1]);
                        acc[4 * k + 2] = fmaf(x, w.z, acc[4 * k + 2]);
                        acc[4 * k + 3] = fmaf(x, w.w, acc[4 * k + 3]);
                    }
                } else {
                    const float4 w4 = *reinterpret_cast<const float4 *>(wt);
                    const float wv[DFT_N2] = {w4.x, w4.y, w4.z, w4.w, wt[4]};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (ser[q] < 0) continue;
                        const float x = xr[ser[q]];
#pragma unroll
                        for (int i = 0; i < DFT_N2; ++i) acc[q * DFT_N2 + i] = fmaf(x, wv[i], acc[q * DFT_N2 + i]);
                    }
                }
            }
        }
        if (g == groups - 1 && lane < nl) {  // the tile's sums are complete: stage them
            float *o = s_out + (size_t)lane * nc;
            if (dens) {
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (d0 + i < n1) o[d0 + i] = acc[i];
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (ser[q] < 0) continue;
#pragma unroll
                    for (int i = 0; i < DFT_N2; ++i) o[n1 + (ser[q] - 1) * DFT_N2 + i] = acc[q * DFT_N2 + i];
                }
            }
        }
        if (g == groups - 1) {
#pragma unroll
            for (int i = 0; i < 20; ++i) acc[i] = 0.0f;
        }
        __syncthreads();  // every thread is done with stage st (and s_out is complete)
        if (threadIdx.x == 0 && unit + DFTB_STAGES < units) issue(unit + DFTB_STAGES);
        if (g == groups - 1)  // written contiguously; s_out is next written a whole tile later
            for (int q = threadIdx.x; q < nl * nc; q += blockDim.x) coeffs[(size_t)leaf0 * nc + q] = s_out[q];
    }
    if (s_fail) {
        // NaN into every coefficient of this CTA's unfinished tiles, then drain
        // the copies in flight (bounded) and report
        const float nan = __int_as_float(0x7fc00000);
        for (uint32_t k = unit / groups; k < my_tiles; ++k) {
            const uint32_t leaf0 = (blockIdx.x + k * gridDim.x) * DFT_TILE;
            const uint32_t nl = min((uint32_t)DFT_TILE, n_leaves - leaf0);
            for (uint32_t q = threadIdx.x; q < nl * (uint32_t)nc; q += blockDim.x) coeffs[(size_t)leaf0 * nc + q] = nan;
        }
        if (threadIdx.x == 0) {
            for (uint32_t u = unit; u < unit + DFTB_STAGES && u < units; ++u)
                ptx::mbar_wait_bounded(&bars[u % DFTB_STAGES], (u / DFTB_STAGES) & 1u, WAIT_LIMIT_NS);
            if (status) atomicOr(status, STATUS_DEVICE_TIMEOUT);
        }
    }
}


int launch_dft(const float *values, float *coeffs, uint32_t n_leaves, int n1, int n2, int T, uint32_t *status,
               bool test_timeout, int sm_count, void *stream)
{
    if (n_leaves == 0) return (int)cudaSuccess;
    // bulk copies need a 16-byte aligned base (every frame row of a tile
    // starts a multiple of 112 bytes further); other bases take the tile kernel
    if (n2 == DFT_N2 && n1 <= 32 && (reinterpret_cast<uintptr_t>(values) & 15u) == 0) {
        const int nc = n1 + 27 * DFT_N2;
        const size_t smem = ((size_t)DFTB_STAGES * DFTB_FPS * DFT_FRAME_FLOATS + (size_t)T * 32 + (size_t)DFT_TILE * nc) *
                            sizeof(float);
        cudaError_t e = cudaFuncSetAttribute(dft_bulk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return (int)e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dft_bulk_kernel, DFTB_THREADS, smem);
        if (e != cudaSuccess) return (int)e;
        if (per_sm < 1) per_sm = 1;
        const uint64_t n_tiles = (n_leaves + DFT_TILE - 1) / DFT_TILE;
        uint64_t blocks = (uint64_t)sm_count * per_sm;
        if (blocks > n_tiles) blocks = n_tiles;
        dft_bulk_kernel<<<(unsigned)blocks, DFTB_THREADS, smem, (cudaStream_t)stream>>>(values, coeffs, n_leaves, n1, T,
                                                                                         status, test_timeout);
        return (int)cudaGetLastError();
    }
    if (n2 == DFT_N2 && n1 <= 32) {
        const int nc = n1 + 27 * DFT_N2;
        const size_t smem = ((size_t)T * 32 + DFT_TC * DFT_TILE * DFT_XPAD + (size_t)DFT_TILE * nc) * sizeof(float);
        cudaError_t e = cudaFuncSetAttribute(dft_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return (int)e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dft_tile_kernel, 256, smem);
        if (e != cudaSuccess) return (int)e;
        if (per_sm < 1) per_sm = 1;
        const uint64_t n_tiles = (n_leaves + DFT_TILE - 1) / DFT_TILE;
        uint64_t blocks = (uint64_t)sm_count * per_sm;
        if (blocks > n_tiles) blocks = n_tiles;
        dft_tile_kernel<<<(unsigned)blocks, 256, smem, (cudaStream_t)stream>>>(values, coeffs, n_leaves, n1, T);
        return (int)cudaGetLastError();
    }
    const uint64_t total = (uint64_t)n_leaves * (n1 + 27 * n2);
    uint64_t blocks = (total + 255) / 256;
    if (blocks > (uint64_t)sm_count * 32) blocks = (uint64_t)sm_count * 32;
    dft_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(values, coeffs, n_leaves, n1, n2, T);
    return (int)cudaGetLastError();
}

}  // namespace fpo
