// Latent decoder on the 5th-generation tensor cores (tcgen05, TMEM).
//
// Each leaf stores a 32-dim FP16 latent; a shared MLP 32 -> 64 -> 64 -> 166
// (ReLU) decodes the leaf's n1 + 27 n2 Fourier coefficients.  Eq. 7 and 9 are
// linear in the coefficients, so the frame's IDFT is folded into the last
// layer: W3'(t) = B(t) W3, b3'(t) = B(t) b3 with B(t) the 28 x 166 map to
// (sigma_raw, z_{c,k}), and the kernel writes the same per-frame table as the
// coefficient IDFT pass: [max(0, sigma), 27 z, 0 x 4] per leaf.
//
// Per CTA the weights are staged once in shared memory in the no-swizzle
// K-major core-matrix layout (8 rows x 16 B blocks) and W3'(t) is computed
// in the prologue.  Eight warpgroups (1024 threads, all 512 TMEM columns)
// then run independent tile pipelines
// (own A buffers, own 64 TMEM columns, own mbarrier and named barrier): for
// each tile of 128 leaves the threads lay the latents out as the A operand,
// one elected thread issues tcgen05.mma (M = 128, K = 16 per instruction,
// FP16 x FP16 -> FP32 in TMEM) and commits to the mbarrier, and the warps
// read the accumulator rows back with tcgen05.ld (one row per thread, a
// warp's TMEM lane quarter), apply ReLU while rounding to FP16 and write the
// next layer's A operand.  The 64 columns hold every layer's accumulator in
// turn.  The output tile goes out by one TMA tensor store per tile.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstdint>

#include "fpo_internal.h"
#include "fpo_ptx.cuh"

namespace fpo {
namespace {

// Independent warpgroup pipelines per CTA (one CTA per SM): 8 (1024 threads,
// all 512 TMEM columns) when the decoder has the SM to itself, 2 (256
// threads, 128 columns) beside the traversal in the frame pipeline.
constexpr int LT_GROUPS_FULL = 8, LT_GROUPS_PIPE = 2;
constexpr int LT_M = 128;          // leaves per tile = MMA M
// 64 accumulator columns per warpgroup
template <int G>
__host__ __device__ constexpr uint32_t lt_tmem_cols() { return 64u * G; }
static_assert(lt_tmem_cols<LT_GROUPS_FULL>() <= 512 && lt_tmem_cols<LT_GROUPS_PIPE>() >= 32, "TMEM allocation");
constexpr uint64_t LT_WAIT_NS = 2000000000ull;

// Biases ride in the MMAs: every A operand carries two constant-one columns
// after its data and every B operand the bias split into two FP16 halves
// (hi = fp16(b), lo = fp16(b - hi), so hi + lo carries b to about 22 bits)
// in the same two columns; the accumulator then already holds W x + b.  K
// is padded to a multiple of 16 with zeros: 32 + 16 for layer 1, 64 + 16 for
// layers 2 and 3.
constexpr int K1 = 48, K2 = 80;

// Shared-memory layout (bytes), all operands no-swizzle K-major.
constexpr int OFF_W1 = 0;          // 64 x 48  f16:  6 KB
constexpr int OFF_W2 = 6144;       // 64 x 80  f16: 10 KB
constexpr int OFF_W3 = 16384;      // 32 x 80  f16:  5 KB
// A1 (layer-1 input) and A2 share one region per group: MMA 1 has finished
// reading A1 before the layer-1 epilogue writes A2, and the next tile's A1 is
// written only after the tensor store has read the previous output from A2.
constexpr int OFF_A1 = 22528;      // per group: 128 x 48 f16: 12 KB
constexpr int OFF_A2 = 22528;      // per group: 128 x 80 f16: 20 KB (1024-byte aligned: output staging)
constexpr int GROUP_BYTES = 20480; // one warpgroup's region
template <int G>
__host__ __device__ constexpr int lt_smem() { return OFF_A1 + G * GROUP_BYTES + 1024; }  // + alignment slack

// Byte offset of element (row, k) in a K-major core-matrix layout whose rows
// hold K elements: core matrix (row / 8, k / 8) at ((row/8) * K/8 + k/8) * 128,
// inside it row % 8 at 16 B per row.
__device__ __forceinline__ uint32_t core_off(int row, int k, int K)
{
    return (uint32_t)((((row >> 3) * (K >> 3) + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// kind::f16 instruction descriptor: A, B f16, D f32, both K-major, M x N.
__device__ __forceinline__ uint32_t idesc_f16(int M, int N)
{
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     ptx::smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 consecutive FP32 columns of this thread's TMEM lane; waits for them.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float v[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Tensor store of a 128-row tile of the table (box 32 floats x 128 rows,
// 128-byte swizzle) from shared memory, committed as its own bulk group.
__device__ __forceinline__ void tensor_store_rows(const CUtensorMap *map, const void *src, uint32_t row0)
{
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];\n\t"
                 "cp.async.bulk.commit_group;" ::"l"(reinterpret_cast<uint64_t>(map)),
                 "r"(0), "r"(row0), "r"(ptx::smem_u32(src))
                 : "memory");
}
// Waits until every committed bulk store has finished reading shared memory.
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// Waits until every committed bulk store has completed.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Rounds 8 consecutive values to FP16 with ReLU (max(x, 0) after rounding
// equals rounding after max) and writes them as K-chunk j of row `row` of a
// core layout.  `hmax` keeps the packed running maximum of what was written:
// a value beyond the FP16 range rounds to +inf, which the maximum keeps.
__device__ __forceinline__ void put8_relu(unsigned char *base, int row, int j, int K, const float *v, __half2 &hmax)
{
    uint32_t h[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {  // the first operand goes to the upper half
        asm("cvt.rn.relu.f16x2.f32 %0, %1, %2;" : "=r"(h[e]) : "f"(v[2 * e + 1]), "f"(v[2 * e]));
        hmax = __hmax2(hmax, *reinterpret_cast<const __half2 *>(&h[e]));
    }
    *reinterpret_cast<uint4 *>(base + core_off(row, 8 * j, K)) = make_uint4(h[0], h[1], h[2], h[3]);
}

constexpr float F16_MAX = 65504.0f;  // the largest finite FP16 value

// Writes 8 consecutive values of row `row` (K-chunk j) into a core layout.
__device__ __forceinline__ void put8(unsigned char *base, int row, int j, int K, const float *v)
{
    __half2 h[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) h[e] = __floats2half2_rn(v[2 * e], v[2 * e + 1]);
    *reinterpret_cast<uint4 *>(base + core_off(row, 8 * j, K)) = *reinterpret_cast<const uint4 *>(h);
}

// K-chunk j of row `row` = {hi(b), lo(b), 0 x 6}: the bias columns of a B
// operand; with `ones`, {1, 1, 0 x 6}: the constant columns of an A operand.
__device__ __forceinline__ void put_bias_chunk(unsigned char *base, int row, int j, int K, float b, bool ones)
{
    const __half hi = ones ? __float2half_rn(1.0f) : __float2half_rn(b);
    const __half lo = ones ? __float2half_rn(1.0f) : __float2half_rn(b - __half2float(hi));
    const __half2 h0 = __halves2half2(hi, lo), z = __float2half2_rn(0.0f);
    uint4 u;
    u.x = *reinterpret_cast<const uint32_t *>(&h0);
    u.y = u.z = u.w = *reinterpret_cast<const uint32_t *>(&z);
    *reinterpret_cast<uint4 *>(base + core_off(row, 8 * j, K)) = u;
}

__device__ __forceinline__ void put_zero_chunk(unsigned char *base, int row, int j, int K)
{
    *reinterpret_cast<uint4 *>(base + core_off(row, 8 * j, K)) = make_uint4(0, 0, 0, 0);
}

// Issues the K / 16 MMAs of D[128 x N] = A[128 x K] B[N x K]^T.
__device__ __forceinline__ void gemm(uint32_t d_tmem, uint32_t a_saddr, uint32_t b_saddr, int K, int N)
{
    const uint32_t idesc = idesc_f16(LT_M, N);
    const uint32_t sbo = (uint32_t)(K / 8) * 128u;
#pragma unroll 1
    for (int s = 0; s < K / 16; ++s) {
        const uint64_t a = smem_desc(a_saddr + 256u * s, 128u, sbo);
        const uint64_t b = smem_desc(b_saddr + 256u * s, 128u, sbo);
        mma_f16(d_tmem, a, b, idesc, s > 0 ? 1u : 0u);
    }
}

}  // namespace

__device__ __forceinline__ void group_sync(int group)
{
    asm volatile("bar.sync %0, 128;" ::"r"(1 + group) : "memory");
}

template <int G>
__global__ void __launch_bounds__(128 * G, 8 / G) latent_table_kernel(const __grid_constant__ LatentParams p)
{
    constexpr int LT_GROUPS = G, LT_THREADS = 128 * G;
    constexpr uint32_t LT_TMEM_COLS = lt_tmem_cols<G>();
    extern __shared__ __align__(1024) unsigned char lt_smem_raw[];
    // the 128-byte-swizzled output staging needs 1024-byte aligned buffers
    unsigned char *lt_smem = lt_smem_raw + ((1024u - (ptx::smem_u32(lt_smem_raw) & 1023u)) & 1023u);
    __shared__ float s_basis[32];
    __shared__ uint64_t s_bar[LT_GROUPS];
    __shared__ uint64_t s_never;  // FPO_FLAG_TEST_DEVICE_TIMEOUT: a barrier nothing signals
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail[LT_GROUPS];
    __shared__ int s_range;  // a weight or bias beyond the FP16 range
    const int tid = threadIdx.x, warp = tid >> 5;
    const int group = tid >> 7, gt = tid & 127;  // warpgroup and thread within it

    // --- prologue: basis, weights (bf16 -> f16, core layout), folded layer 3
    const int nb = p.n1 > p.n2 ? p.n1 : p.n2;
    if (tid < 32) s_basis[tid] = tid < nb ? (float)((tid & 1) ? sinpi((double)(tid + 1) * (p.t / p.period_T))
                                                             : cospi((double)tid * (p.t / p.period_T)))
                                         : 0.0f;
    if (tid == 0) s_range = 0;
    if (tid < LT_GROUPS) {
        s_fail[tid] = 0;
        ptx::mbar_init(&s_bar[tid], 1);
        if (tid == 0) ptx::mbar_init(&s_never, 1);
        ptx::fence_barrier_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(ptx::smem_u32(&s_tmem)),
                     "r"(LT_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int q = tid; q < 64 * (K1 / 8); q += LT_THREADS) {  // W1 | b1: 64 rows x 6 chunks
        const int n = q / (K1 / 8), j = q % (K1 / 8);
        if (j < 4) {
            float v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = __bfloat162float(__ushort_as_bfloat16(p.w1[n * 32 + 8 * j + e]));
            for (int e = 0; e < 8; ++e)
                if (!(fabsf(v[e]) <= F16_MAX)) s_range = 1;
            put8(lt_smem + OFF_W1, n, j, K1, v);
        } else if (j == 4) {
            if (!(fabsf(p.b1[n]) <= F16_MAX)) s_range = 1;
            put_bias_chunk(lt_smem + OFF_W1, n, j, K1, p.b1[n], false);
        } else {
            put_zero_chunk(lt_smem + OFF_W1, n, j, K1);
        }
    }
    for (int q = tid; q < 64 * (K2 / 8); q += LT_THREADS) {  // W2 | b2: 64 rows x 10 chunks
        const int n = q / (K2 / 8), j = q % (K2 / 8);
        if (j < 8) {
            float v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = __bfloat162float(__ushort_as_bfloat16(p.w2[n * 64 + 8 * j + e]));
            for (int e = 0; e < 8; ++e)
                if (!(fabsf(v[e]) <= F16_MAX)) s_range = 1;
            put8(lt_smem + OFF_W2, n, j, K2, v);
        } else if (j == 8) {
            if (!(fabsf(p.b2[n]) <= F16_MAX)) s_range = 1;
            put_bias_chunk(lt_smem + OFF_W2, n, j, K2, p.b2[n], false);
        } else {
            put_zero_chunk(lt_smem + OFF_W2, n, j, K2);
        }
    }
    __syncthreads();  // s_basis ready
    // W3'(t): row 0 = sum_i b_i W3[i], row 1 + q = sum_i b_i W3[n1 + q n2 + i],
    // rows 28..31 = 0.  One output element per thread and pass: the loads of a
    // row are coalesced over h and independent of each other (unrolled), so
    // the prologue costs a few memory latencies, not one per term.
    for (int q = tid; q < 32 * 64; q += LT_THREADS) {
        const int r = q >> 6, h = q & 63;
        const int row0 = r == 0 ? 0 : p.n1 + (r - 1) * p.n2, terms = r == 0 ? p.n1 : (r <= 27 ? p.n2 : 0);
        float acc = 0.0f;
#pragma unroll 8
        for (int i = 0; i < terms; ++i)
            acc = fmaf(s_basis[i], __bfloat162float(__ushort_as_bfloat16(p.w3[(row0 + i) * 64 + h])), acc);
        if (!(fabsf(acc) <= F16_MAX)) s_range = 1;
        *reinterpret_cast<__half *>(lt_smem + OFF_W3 + core_off(r, h, K2)) = __float2half_rn(acc);
    }
    if (tid < 32) {
        const int row0 = tid == 0 ? 0 : p.n1 + (tid - 1) * p.n2, terms = tid == 0 ? p.n1 : (tid <= 27 ? p.n2 : 0);
        float acc = 0.0f;
#pragma unroll 8
        for (int i = 0; i < terms; ++i) acc = fmaf(s_basis[i], p.b3[row0 + i], acc);
        if (!(fabsf(acc) <= F16_MAX)) s_range = 1;
        put_bias_chunk(lt_smem + OFF_W3, tid, 8, K2, acc, false);  // rows 28..31: b = 0
        put_zero_chunk(lt_smem + OFF_W3, tid, 9, K2);
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    // this warpgroup's accumulator columns; this warp's lane quarter
    const uint32_t tmem = s_tmem + 64u * (uint32_t)group;
    const uint32_t my_lane = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    unsigned char *ga1 = lt_smem + OFF_A1 + group * GROUP_BYTES;
    unsigned char *ga2 = lt_smem + OFF_A2 + group * GROUP_BYTES;
    const uint32_t sa_w1 = ptx::smem_u32(lt_smem + OFF_W1), sa_w2 = ptx::smem_u32(lt_smem + OFF_W2),
                   sa_w3 = ptx::smem_u32(lt_smem + OFF_W3), sa_a1 = ptx::smem_u32(ga1), sa_a2 = ptx::smem_u32(ga2);
    uint32_t phase = 0;
    __half2 hmax = __float2half2_rn(0.0f);  // packed maximum of the FP16 activations written
    const uint32_t n_tiles = (p.n_leaves + LT_M - 1) / LT_M;
    const uint32_t first = blockIdx.x * LT_GROUPS + group, step = gridDim.x * LT_GROUPS;
    const int m = gt;  // this thread's accumulator row (TMEM lane) and leaf in the tile


    // One layer: the group's elected thread issues the MMAs and commits;
    // the group waits on its mbarrier (bounded).  The outcome is made
    // group-uniform so that the collective TMEM loads never diverge.  On a
    // time-out `phase` stays at the pending commit, which the drain after
    // the loop waits for before TMEM is freed.  The failure-path test makes
    // the group's first wait (on a barrier nothing signals) run out.
    bool first_wait = p.test_timeout != 0;
    auto run_layer = [&](uint32_t a_addr, uint32_t b_addr, int K, int N) -> bool {
        if (gt == 0) {
            fence_after();
            gemm(tmem, a_addr, b_addr, K, N);
            mma_commit(&s_bar[group]);
        }
        const bool ok = first_wait ? ptx::mbar_wait_bounded(&s_never, 0, TEST_WAIT_LIMIT_NS)
                                   : ptx::mbar_wait_bounded(&s_bar[group], phase, LT_WAIT_NS);
        first_wait = false;
        if (!ok) s_fail[group] = 1;
        group_sync(group);
        fence_after();
        if (s_fail[group]) return false;
        phase ^= 1u;
        return true;
    };
    auto hand_off = [&]() {  // generic smem writes and TMEM reads before the next MMA
        fence_async_smem();
        fence_before();
        group_sync(group);
    };
    // The tile's latents (128 rows x 64 B, contiguous) in coalesced 16-byte
    // pieces: thread gt takes pieces gt + 128 i, i.e. row (gt + 128 i) / 4,
    // K-chunk (gt + 128 i) % 4; rows past the end read as zeros.
    auto load_tile = [&](uint32_t tile, uint4 q[4]) {
        const uint4 *src = reinterpret_cast<const uint4 *>(p.latents) + (size_t)tile * LT_M * 4;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int piece = gt + 128 * i;
            q[i] = make_uint4(0, 0, 0, 0);
            if (tile < n_tiles && tile * LT_M + (uint32_t)(piece >> 2) < p.n_leaves) q[i] = __ldg(src + piece);
        }
    };
    uint4 nextq[4];
    load_tile(first, nextq);
    for (uint32_t tile = first; tile < n_tiles; tile += step) {
        if (gt == 0) bulk_wait_read();  // the previous tile's table store has left A2
        group_sync(group);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int piece = gt + 128 * i;
            *reinterpret_cast<uint4 *>(ga1 + core_off(piece >> 2, 8 * (piece & 3), K1)) = nextq[i];
        }
        // the constant-one columns of this thread's row (A2 writes reuse the region)
        put_bias_chunk(ga1, m, 4, K1, 0.0f, true);
        put_zero_chunk(ga1, m, 5, K1);
        hand_off();
        if (!run_layer(sa_a1, sa_w1, K1, 64)) break;
        // layer 1 epilogue: bias + ReLU -> layer-2 A operand (MMA 1 is done with A1)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float v[32];
            tmem_ld32(my_lane + 32 * h, v);
#pragma unroll
            for (int c = 0; c < 4; ++c) put8_relu(ga2, m, 4 * h + c, K2, v + 8 * c, hmax);
        }
        put_bias_chunk(ga2, m, 8, K2, 0.0f, true);
        put_zero_chunk(ga2, m, 9, K2);
        hand_off();
        if (!run_layer(sa_a2, sa_w2, K2, 64)) break;
        // layer 2 epilogue -> layer-3 A operand, in place (MMA 2 has finished
        // reading A2, and each thread rewrites only its own row)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float v[32];
            tmem_ld32(my_lane + 32 * h, v);
#pragma unroll
            for (int c = 0; c < 4; ++c) put8_relu(ga2, m, 4 * h + c, K2, v + 8 * c, hmax);
        }
        hand_off();
        load_tile(tile + step, nextq);  // in flight while layer 3 runs
        if (!run_layer(sa_a2, sa_w3, K2, 32)) break;
        {
            // output rows [max(0, sigma), 27 z, 0 x 4] into A2 (free since MMA 3
            // finished), then one bulk copy of the tile's contiguous rows
            float o[32];
            tmem_ld32(my_lane, o);
            // the accumulator holds W3'x + b3': sigma gets its clamp, columns
            // 28..31 are exactly zero
            float *w = o;
            w[0] = fmaxf(w[0], 0.0f);
            // 128-byte swizzle (chunk q of row m at chunk q ^ (m % 8)): the 8
            // lanes of a store phase hit 8 different bank groups, and the
            // tensor store un-swizzles on the way out
            if (p.half_table) {
                // FP16 rows of 64 B with the 64-byte swizzle (chunk q of row m
                // at chunk q ^ ((m / 2) % 4)): again no bank conflicts
                uint4 *row = reinterpret_cast<uint4 *>(ga2 + m * (TABLE_STRIDE * 2));
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    uint32_t h[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const __half2 hh = __floats2half2_rn(w[8 * q + 2 * e], w[8 * q + 2 * e + 1]);
                        h[e] = *reinterpret_cast<const uint32_t *>(&hh);
                    }
                    row[q ^ ((m >> 1) & 3)] = make_uint4(h[0], h[1], h[2], h[3]);
                }
            } else {
                float4 *row = reinterpret_cast<float4 *>(ga2 + m * (TABLE_STRIDE * 4));
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    row[q ^ (m & 7)] = make_float4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
            }
        }
        fence_async_smem();
        fence_before();
        group_sync(group);  // the rows are in A2; the accumulator is free for the next tile
        if (gt == 0) tensor_store_rows(&p.table_map, ga2, tile * LT_M);  // rows past the end are clipped
    }
    if (gt == 0) bulk_wait_all();  // every table store has completed
    // FP16 operands: a hidden activation, weight or bias beyond the FP16
    // range (it became +inf) makes the table wrong; report it
    if (p.status && (!(__low2float(hmax) <= F16_MAX) || !(__high2float(hmax) <= F16_MAX) || (tid == 0 && s_range)))
        atomicOr(p.status, STATUS_FP16_RANGE);
    if (s_fail[group] && gt == 0) {
        // the commit whose wait gave up: wait for it once more (bounded)
        // before TMEM is freed
        ptx::mbar_wait_bounded(&s_bar[group], phase, LT_WAIT_NS);
        if (p.status) atomicOr(p.status, STATUS_DEVICE_TIMEOUT);
    }
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_tmem), "r"(LT_TMEM_COLS) : "memory");
}

// ---------------------------------------------------------------------------
// Tensor-core training step of the decoder: the forward pass, the weighted L2
// loss against target coefficients (plus an optional extra dL/dy), and the
// back-propagation to every weight, bias and latent, with BF16 operands (A
// and B of each MMA both BF16; FP32's exponent range, so no loss scaling)
// and FP32 accumulation in TMEM.  One warpgroup per CTA and one CTA per SM
// (all 512 TMEM columns); thread t owns row t of a 128-leaf tile and TMEM
// lane t.  Per tile, nine GEMMs (M = 128, no-swizzle K-major operands):
//   Z1 = [X 1] W1'^T,  Z2 = [H1 1] W2'^T,  Y = [H2 1] W3'^T       (forward)
//   dH2 = dY W3,  dH1 = d2 W2,  dX = d1 W1                        (data)
//   G3 += [H2^T; 1] dY,  G2 += [H1^T; 1] d2,  G1 += [X^T; 1] d1    (weights)
// H = relu(Z) in BF16, d2 = dH2 [Z2 > 0], d1 = dH1 [Z1 > 0], dY = 2 cw (Y -
// target) + extra.  The weight gradients accumulate in TMEM over all of the
// CTA's tiles, transposed (lane = input feature, column = output feature);
// the ones row of each transposed activation makes lane 64 (32 for layer 1)
// the bias gradient.  The transposed operands (activations and gradients
// with the tile's rows as K) are written by the epilogues next to the
// row-major ones.  The M = 128 A operands of the weight GEMMs hold only
// 40 or 72 meaningful rows; the rest of each descriptor's extent reads
// whatever lies after them in shared memory, which lands only in TMEM lanes
// that are never read.
namespace {

constexpr int TG_K1 = 48, TG_K2 = 80, TG_NC = 176, TG_KR = 128;
constexpr int TGO_W1 = 0;                          // [64][48]   W1 | b1 (B of Z1)
constexpr int TGO_W2 = TGO_W1 + 64 * TG_K1 * 2;    // [64][80]   W2 | b2 (B of Z2)
constexpr int TGO_W3 = TGO_W2 + 64 * TG_K2 * 2;    // [176][80]  W3 | b3 (B of Y)
constexpr int TGO_W3T = TGO_W3 + TG_NC * TG_K2 * 2;  // [64][176] W3^T (B of dH2)
constexpr int TGO_W2T = TGO_W3T + 64 * TG_NC * 2;  // [64][64]   W2^T (B of dH1)
constexpr int TGO_W1T = TGO_W2T + 64 * 64 * 2;     // [32][64]   W1^T (B of dX)
constexpr int TGO_XT = TGO_W1T + 32 * 64 * 2;      // [40][128]  [X^T; 1] (A of G1)
constexpr int TGO_H1T = TGO_XT + 40 * TG_KR * 2;   // [72][128]  [H1^T; 1] (A of G2)
constexpr int TGO_H2T = TGO_H1T + 72 * TG_KR * 2;  // [72][128]  [H2^T; 1] (A of G3)
constexpr int TGO_A = TGO_H2T + 72 * TG_KR * 2;    // the tile's A operand: [X 1], [H1 1], [H2 1], dY, d2, d1
constexpr int TGO_B = TGO_A + 128 * TG_NC * 2;     // the weight GEMMs' B operand: dY^T, d2^T, d1^T
constexpr int TG_SMEM = TGO_B + TG_NC * TG_KR * 2;
static_assert(TGO_XT + 128 * TG_KR * 2 <= TG_SMEM && TGO_H2T + 128 * TG_KR * 2 <= TG_SMEM,
              "the weight GEMMs' A descriptors stay inside the CTA's shared memory");
// TMEM columns: per-tile scratch (Z1, Z2, Y, dH2, dH1, dX) and the weight gradients
constexpr uint32_t TC_SCR = 0, TC_G3 = 192, TC_G2 = 384, TC_G1 = 448, TC_COLS = 512;

struct DecoderGradTcParams {
    fpo_mlp w, g;
    const uint32_t *rows;
    uint32_t batch;
    const float *latents, *targets, *coef_weight, *extra_dy;
    float *dlatents;
    double *loss;
    uint32_t *status;
    int nc;
    int test_timeout;
};

__device__ __forceinline__ uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D[128 x N] (+)= A[128 x K] B[N x K]^T, BF16; acc0: accumulate from the first K slice on.
__device__ __forceinline__ void gemm_bf16(uint32_t d_tmem, uint32_t a_saddr, uint32_t b_saddr, int K, int N,
                                          uint32_t acc0)
{
    const uint32_t idesc = idesc_bf16(128, N);
    const uint32_t sbo = (uint32_t)(K / 8) * 128u;
#pragma unroll 1
    for (int s = 0; s < K / 16; ++s) {
        const uint64_t a = smem_desc(a_saddr + 256u * s, 128u, sbo);
        const uint64_t b = smem_desc(b_saddr + 256u * s, 128u, sbo);
        mma_f16(d_tmem, a, b, idesc, s > 0 ? 1u : acc0);
    }
}

__device__ __forceinline__ void put1_bf(unsigned char *base, int row, int k, int K, float v)
{
    *reinterpret_cast<__nv_bfloat16 *>(base + core_off(row, k, K)) = __float2bfloat16_rn(v);
}

// 8 consecutive values of row `row` (K-chunk j) as BF16.
__device__ __forceinline__ void put8_bf(unsigned char *base, int row, int j, int K, const float *v)
{
    uint32_t h[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
        h[e] = *reinterpret_cast<const uint32_t *>(&b);
    }
    *reinterpret_cast<uint4 *>(base + core_off(row, 8 * j, K)) = make_uint4(h[0], h[1], h[2], h[3]);
}

// K-chunk j of row `row` = {hi(b), lo(b), 0 x 6} in BF16 (hi + lo carries b
// to about 16 bits), or {c, c, 0 x 6}: the constant columns of an A operand.
__device__ __forceinline__ void put_pair_bf(unsigned char *base, int row, int j, int K, float a, float b)
{
    const __nv_bfloat162 p = __floats2bfloat162_rn(a, b);
    *reinterpret_cast<uint4 *>(base + core_off(row, 8 * j, K)) =
        make_uint4(*reinterpret_cast<const uint32_t *>(&p), 0u, 0u, 0u);
}
__device__ __forceinline__ void put_bias_bf(unsigned char *base, int row, int j, int K, float b)
{
    const float hi = __bfloat162float(__float2bfloat16_rn(b));
    put_pair_bf(base, row, j, K, hi, b - hi);
}

// Rows owned by the lanes of a warp (lane r: row offset off_r, validity ok_r)
// moved in coalesced pieces through a per-warp shared tile of H rows x 33
// floats: for each row, the 32 lanes move 32 consecutive floats (columns col0
// + lane, those below ncols), and the tile turns them into each lane's own
// 32 values (H = 32: one pass; H = 16: two passes of half the rows).
template <int H>
__device__ __forceinline__ void warp_load_rows(float v[32], const float *__restrict__ base, size_t off, bool ok,
                                               int col0, int ncols, float *tile)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int h = 0; h < 32 / H; ++h) {
#pragma unroll 4
        for (int i = 0; i < H; ++i) {
            const int r = H * h + i;
            const size_t o = __shfl_sync(0xffffffffu, off, r);
            const bool k = __shfl_sync(0xffffffffu, ok, r);
            const int c = col0 + lane;
            tile[i * 33 + lane] = k && c < ncols ? base[o + c] : 0.0f;
        }
        __syncwarp();
        if ((lane / H) == h) {
#pragma unroll
            for (int e = 0; e < 32; ++e) v[e] = tile[(lane - H * h) * 33 + e];
        }
        __syncwarp();
    }
}

// The inverse: each lane's 32 values of its row to columns col0 + e (those
// below ncols) of its row, where a column j goes to base_lo[off_lo + j] for
// j < split and to base_hi[off_hi + j - split] otherwise (H as above).
template <int H>
__device__ __forceinline__ void warp_store_rows(const float v[32], float *base_lo, size_t off_lo, float *base_hi,
                                                size_t off_hi, int split, bool ok, int col0, int ncols, float *tile)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int h = 0; h < 32 / H; ++h) {
        if ((lane / H) == h) {
#pragma unroll
            for (int e = 0; e < 32; ++e) tile[(lane - H * h) * 33 + e] = v[e];
        }
        __syncwarp();
#pragma unroll 4
        for (int i = 0; i < H; ++i) {
            const int r = H * h + i;
            const size_t olo = __shfl_sync(0xffffffffu, off_lo, r), ohi = __shfl_sync(0xffffffffu, off_hi, r);
            const bool k = __shfl_sync(0xffffffffu, ok, r);
            const int c = col0 + lane;
            if (k && c < ncols) {
                const float x = tile[i * 33 + lane];
                if (c < split) base_lo[olo + c] = x;
                else base_hi[ohi + c - split] = x;
            }
        }
        __syncwarp();
    }
}

}  // namespace

__global__ void __launch_bounds__(128, 1) decoder_grad_tc_kernel(const __grid_constant__ DecoderGradTcParams p)
{
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ uint64_t s_bar, s_never;
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    __shared__ double s_loss;
    const int t = threadIdx.x, warp = t >> 5;
    const int nc = p.nc;
    if (t == 0) {
        s_fail = 0;
        s_loss = 0.0;
        ptx::mbar_init(&s_bar, 1);
        ptx::mbar_init(&s_never, 1);
        ptx::fence_barrier_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(ptx::smem_u32(&s_tmem)),
                     "r"(TC_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // --- weights as BF16 B operands, once per CTA
    for (int q = t; q < 64 * (TG_K1 / 8); q += 128) {
        const int n = q / (TG_K1 / 8), j = q % (TG_K1 / 8);
        if (j < 4) put8_bf(sm + TGO_W1, n, j, TG_K1, p.w.w1 + n * 32 + 8 * j);
        else if (j == 4) put_bias_bf(sm + TGO_W1, n, j, TG_K1, p.w.b1[n]);
        else put_pair_bf(sm + TGO_W1, n, j, TG_K1, 0.0f, 0.0f);
    }
    for (int q = t; q < 64 * (TG_K2 / 8); q += 128) {
        const int n = q / (TG_K2 / 8), j = q % (TG_K2 / 8);
        if (j < 8) put8_bf(sm + TGO_W2, n, j, TG_K2, p.w.w2 + n * 64 + 8 * j);
        else if (j == 8) put_bias_bf(sm + TGO_W2, n, j, TG_K2, p.w.b2[n]);
        else put_pair_bf(sm + TGO_W2, n, j, TG_K2, 0.0f, 0.0f);
    }
    for (int q = t; q < TG_NC * (TG_K2 / 8); q += 128) {
        const int n = q / (TG_K2 / 8), j = q % (TG_K2 / 8);
        if (n >= nc || j == 9) put_pair_bf(sm + TGO_W3, n, j, TG_K2, 0.0f, 0.0f);
        else if (j < 8) put8_bf(sm + TGO_W3, n, j, TG_K2, p.w.w3 + n * 64 + 8 * j);
        else put_bias_bf(sm + TGO_W3, n, j, TG_K2, p.w.b3[n]);
    }
    for (int q = t; q < 64 * TG_NC; q += 128) {  // W3^T[k][j] = W3[j][k]
        const int k = q / TG_NC, j = q % TG_NC;
        put1_bf(sm + TGO_W3T, k, j, TG_NC, j < nc ? p.w.w3[j * 64 + k] : 0.0f);
    }
    for (int q = t; q < 64 * 64; q += 128) {  // W2^T[k][o] = W2[o][k]
        const int k = q >> 6, o = q & 63;
        put1_bf(sm + TGO_W2T, k, o, 64, p.w.w2[o * 64 + k]);
    }
    for (int q = t; q < 32 * 64; q += 128) {  // W1^T[k][o] = W1[o][k]
        const int k = q >> 6, o = q & 63;
        put1_bf(sm + TGO_W1T, k, o, 64, p.w.w1[o * 32 + k]);
    }
    // the transposed activations' rows past the ones row, inside their allocation
    for (int q = t; q < 7 * TG_KR; q += 128) {
        put1_bf(sm + TGO_XT, 33 + q / TG_KR, q % TG_KR, TG_KR, 0.0f);
        put1_bf(sm + TGO_H1T, 65 + q / TG_KR, q % TG_KR, TG_KR, 0.0f);
        put1_bf(sm + TGO_H2T, 65 + q / TG_KR, q % TG_KR, TG_KR, 0.0f);
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();

    const uint32_t tm = s_tmem;
    const uint32_t lane_off = (uint32_t)(warp * 32) << 16;  // this warp's lane quarter
    const uint32_t sa = ptx::smem_u32(sm);
    uint32_t phase = 0;
    bool first_wait = p.test_timeout != 0;
    auto hand_off = [&]() {  // generic smem writes and TMEM reads before the next MMAs
        fence_async_smem();
        fence_before();
        __syncthreads();
    };
    auto wait_mmas = [&]() -> bool {  // bounded; CTA-uniform outcome
        const bool ok = first_wait ? ptx::mbar_wait_bounded(&s_never, 0, TEST_WAIT_LIMIT_NS)
                                   : ptx::mbar_wait_bounded(&s_bar, phase, LT_WAIT_NS);
        first_wait = false;
        if (!ok) s_fail = 1;
        __syncthreads();
        fence_after();
        if (s_fail) return false;
        phase ^= 1u;
        return true;
    };
    const uint32_t n_tiles = (p.batch + 127) / 128;
    float lsum = 0.0f;
    uint32_t acc_w = 0;  // the weight gradients accumulate from the CTA's second tile on
    for (uint32_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const uint32_t r0 = tile * 128;
        const bool valid = r0 + (uint32_t)t < p.batch;
        const size_t row = valid ? p.rows[r0 + t] : 0;
        const float one = valid ? 1.0f : 0.0f;
        // X: [x 1] (A of Z1) and [X^T; 1] (A of G1)
        {
            float x[32];
#pragma unroll
            for (int k = 0; k < 32; ++k) x[k] = valid ? p.latents[row * 32 + k] : 0.0f;
#pragma unroll
            for (int j = 0; j < 4; ++j) put8_bf(sm + TGO_A, t, j, TG_K1, x + 8 * j);
            put_pair_bf(sm + TGO_A, t, 4, TG_K1, one, one);
            put_pair_bf(sm + TGO_A, t, 5, TG_K1, 0.0f, 0.0f);
#pragma unroll
            for (int k = 0; k < 32; ++k) put1_bf(sm + TGO_XT, k, t, TG_KR, x[k]);
            put1_bf(sm + TGO_XT, 32, t, TG_KR, one);
        }
        hand_off();
        if (t == 0) {
            fence_after();
            gemm_bf16(tm + TC_SCR, sa + TGO_A, sa + TGO_W1, TG_K1, 64, 0);
            mma_commit(&s_bar);
        }
        if (!wait_mmas()) break;
        // H1 = relu(Z1): [H1 1] (A of Z2), [H1^T; 1] (A of G2), the mask of Z1 > 0
        uint32_t m1[2], m2[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float v[32];
            tmem_ld32(tm + lane_off + TC_SCR + 32 * h, v);
            m1[h] = 0;
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                if (v[e] > 0.0f) m1[h] |= 1u << e;
                v[e] = fmaxf(v[e], 0.0f);
                put1_bf(sm + TGO_H1T, 32 * h + e, t, TG_KR, v[e]);
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) put8_bf(sm + TGO_A, t, 4 * h + c, TG_K2, v + 8 * c);
        }
        put_pair_bf(sm + TGO_A, t, 8, TG_K2, one, one);
        put_pair_bf(sm + TGO_A, t, 9, TG_K2, 0.0f, 0.0f);
        put1_bf(sm + TGO_H1T, 64, t, TG_KR, one);
        hand_off();
        if (t == 0) {
            fence_after();
            gemm_bf16(tm + TC_SCR, sa + TGO_A, sa + TGO_W2, TG_K2, 64, 0);
            mma_commit(&s_bar);
        }
        if (!wait_mmas()) break;
        // H2 = relu(Z2) in place of H1 (Z2 is done with it)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float v[32];
            tmem_ld32(tm + lane_off + TC_SCR + 32 * h, v);
            m2[h] = 0;
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                if (v[e] > 0.0f) m2[h] |= 1u << e;
                v[e] = fmaxf(v[e], 0.0f);
                put1_bf(sm + TGO_H2T, 32 * h + e, t, TG_KR, v[e]);
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) put8_bf(sm + TGO_A, t, 4 * h + c, TG_K2, v + 8 * c);
        }
        put1_bf(sm + TGO_H2T, 64, t, TG_KR, one);
        hand_off();
        if (t == 0) {
            fence_after();
            gemm_bf16(tm + TC_SCR, sa + TGO_A, sa + TGO_W3, TG_K2, TG_NC, 0);
            mma_commit(&s_bar);
        }
        if (!wait_mmas()) break;
        // dY = 2 cw (Y - target) + extra: dY (A of dH2, over the H2 it replaces) and dY^T (B of G3)
#pragma unroll 1
        for (int c = 0; c < TG_NC / 32 + 1; ++c) {
            float v[32];
            tmem_ld32(tm + lane_off + TC_SCR + 32 * c, v);  // columns 176..191: unused scratch
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                const int j = 32 * c + e;
                float d = 0.0f;
                if (valid && j < nc) {
                    const float err = v[e] - p.targets[row * nc + j];
                    const float cw = p.coef_weight[j];
                    lsum = fmaf(cw * err, err, lsum);
                    d = 2.0f * cw * err;
                    if (p.extra_dy) d += p.extra_dy[row * nc + j];
                }
                v[e] = d;
                if (j < TG_NC) put1_bf(sm + TGO_B, j, t, TG_KR, d);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (4 * c + q < TG_NC / 8) put8_bf(sm + TGO_A, t, 4 * c + q, TG_NC, v + 8 * q);
        }
        hand_off();
        if (t == 0) {
            fence_after();
            gemm_bf16(tm + TC_SCR, sa + TGO_A, sa + TGO_W3T, TG_NC, 64, 0);
            gemm_bf16(tm + TC_G3, sa + TGO_H2T, sa + TGO_B, TG_KR, TG_NC, acc_w);
            mma_commit(&s_bar);
        }
        if (!wait_mmas()) break;
        // d2 = dH2 [Z2 > 0]: A of dH1 (over dY) and d2^T (B of G2, over dY^T)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float v[32];
            tmem_ld32(tm + lane_off + TC_SCR + 32 * h, v);
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                v[e] = (m2[h] >> e) & 1u ? v[e] : 0.0f;
                put1_bf(sm + TGO_B, 32 * h + e, t, TG_KR, v[e]);
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) put8_bf(sm + TGO_A, t, 4 * h + c, 64, v + 8 * c);
        }
        hand_off();
        if (t == 0) {
            fence_after();
            gemm_bf16(tm + TC_SCR, sa + TGO_A, sa + TGO_W2T, 64, 64, 0);
            gemm_bf16(tm + TC_G2, sa + TGO_H1T, sa + TGO_B, TG_KR, 64, acc_w);
            mma_commit(&s_bar);
        }
        if (!wait_mmas()) break;
        // d1 = dH1 [Z1 > 0]: A of dX and d1^T (B of G1)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float v[32];
            tmem_ld32(tm + lane_off + TC_SCR + 32 * h, v);
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                v[e] = (m1[h] >> e) & 1u ? v[e] : 0.0f;
                put1_bf(sm + TGO_B, 32 * h + e, t, TG_KR, v[e]);
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) put8_bf(sm + TGO_A, t, 4 * h + c, 64, v + 8 * c);
        }
        hand_off();
        if (t == 0) {
            fence_after();
            gemm_bf16(tm + TC_SCR, sa + TGO_A, sa + TGO_W1T, 64, 32, 0);
            gemm_bf16(tm + TC_G1, sa + TGO_XT, sa + TGO_B, TG_KR, 64, acc_w);
            mma_commit(&s_bar);
        }
        if (!wait_mmas()) break;
        // dL/d(latent) of the tile's rows
        {
            float v[32];
            tmem_ld32(tm + lane_off + TC_SCR, v);
            if (valid) {  // (scalar stores: the caller's array needs only float alignment)
#pragma unroll
                for (int k = 0; k < 32; ++k) p.dlatents[(size_t)(r0 + t) * 32 + k] = v[k];
            }
        }
        fence_before();  // TMEM reads done before the next tile's MMAs
        acc_w = 1;
    }
    if (!s_fail) {
        // the weight gradients: lane k of G3 / G2 / G1 is input feature k, lane
        // 64 (32 for G1) the bias; column j / o the output feature
#pragma unroll 1
        for (int c = 0; c < TG_NC / 32 + 1; ++c) {
            float v[32];
            tmem_ld32(tm + lane_off + TC_G3 + 32 * c, v);  // columns past 175 belong to G3's padding
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                const int j = 32 * c + e;
                if (j >= nc) continue;
                if (t < 64) atomicAdd(p.g.w3 + j * 64 + t, v[e]);
                else if (t == 64) atomicAdd(p.g.b3 + j, v[e]);
            }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float v[32];
            tmem_ld32(tm + lane_off + TC_G2 + 32 * h, v);
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                const int o = 32 * h + e;
                if (t < 64) atomicAdd(p.g.w2 + o * 64 + t, v[e]);
                else if (t == 64) atomicAdd(p.g.b2 + o, v[e]);
            }
            tmem_ld32(tm + lane_off + TC_G1 + 32 * h, v);
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                const int o = 32 * h + e;
                if (t < 32) atomicAdd(p.g.w1 + o * 32 + t, v[e]);
                else if (t == 32) atomicAdd(p.g.b1 + o, v[e]);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
        if ((t & 31) == 0) atomicAdd(&s_loss, (double)lsum);
    } else if (t == 0) {
        // the commit whose wait gave up: wait for it once more (bounded)
        // before TMEM is freed
        ptx::mbar_wait_bounded(&s_bar, phase, LT_WAIT_NS);
        if (p.status) atomicOr(p.status, STATUS_DEVICE_TIMEOUT);
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (t == 0 && p.loss && !s_fail) atomicAdd(p.loss, s_loss);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_tmem), "r"(TC_COLS) : "memory");
}

// ---------------------------------------------------------------------------
// Decode of every leaf into a render context's FP32 records on the tensor
// cores, with the numerics of the inference decoder (FP16 latents, weights
// rounded to BF16 and then FP16, FP16 hidden activations, biases as FP16
// hi/lo pairs, FP32 accumulation) but the last layer unfolded (all
// n1 + 27 n2 coefficients): what the pixel loss of the decoder's training
// renders.  DR_GROUPS independent warpgroup pipelines per CTA, one CTA per SM,
// each with 96 TMEM columns (Z1 and Z2 in the first 64; the last layer in two
// halves, columns 0..95 and 96..175 of Y, each in the 96) and one
// shared-memory region for its tile's A operands; the next tile's latents
// are gathered while the last layer runs.  Tile rows are records: row
// i gathers latent perm[i] and writes record i (density values at stride ss,
// SH values at stride zs).
namespace {
constexpr int DR_GROUPS = 4, DR_NC = 176, DR_COLS = 96, DR_NH0 = 96, DR_NH1 = DR_NC - DR_NH0;
constexpr int DRO_W1 = 0;                        // [64][48]  W1 | b1
constexpr int DRO_W2 = DRO_W1 + 64 * K1 * 2;     // [64][80]  W2 | b2
constexpr int DRO_W3 = DRO_W2 + 64 * K2 * 2;     // [176][80] W3 | b3
constexpr int DRO_A = DRO_W3 + DR_NC * K2 * 2;   // per group: [128][80] (X, then H1, then H2)
constexpr int DR_GROUP_BYTES = 128 * K2 * 2;
constexpr int DRO_ROWS = DRO_A + DR_GROUPS * DR_GROUP_BYTES;  // per warp: 32 x 33 floats
constexpr int DR_SMEM = DRO_ROWS + DR_GROUPS * 4 * 32 * 33 * 4;

struct DecodeTcParams {
    fpo_mlp w;                  // FP32 master weights
    const float *latents;       // [n][32] FP32, upload order
    const uint32_t *perm;       // record -> latent row
    float *sig, *zc;            // FP32 records
    uint32_t n;
    int n1, nc, ss, zs;
    uint32_t *status;
    int test_timeout;
};
}  // namespace

__global__ void __launch_bounds__(128 * DR_GROUPS, 1) decode_records_tc_kernel(const __grid_constant__ DecodeTcParams p)
{
    extern __shared__ __align__(1024) unsigned char dr_smem_raw[];
    unsigned char *sm = dr_smem_raw + ((1024u - (ptx::smem_u32(dr_smem_raw) & 1023u)) & 1023u);
    __shared__ uint64_t s_bar[DR_GROUPS];
    __shared__ uint64_t s_never;
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail[DR_GROUPS];
    __shared__ int s_range;
    const int tid = threadIdx.x, warp = tid >> 5, group = tid >> 7, m = tid & 127;
    const int nc = p.nc;
    if (tid == 0) {
        s_range = 0;
        for (int g = 0; g < DR_GROUPS; ++g) {
            s_fail[g] = 0;
            ptx::mbar_init(&s_bar[g], 1);
        }
        ptx::mbar_init(&s_never, 1);
        ptx::fence_barrier_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(ptx::smem_u32(&s_tmem)),
                     "r"(512u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // weights as FP16 B operands, through BF16 as the inference decoder holds
    // them (values beyond the FP16 range are reported)
    auto wv = [&](float x) {
        x = __bfloat162float(__float2bfloat16_rn(x));
        if (!(fabsf(x) <= F16_MAX)) s_range = 1;
        return x;
    };
    auto bv = [&](float x) {  // biases stay FP32 (an FP16 hi/lo pair in the operand)
        if (!(fabsf(x) <= F16_MAX)) s_range = 1;
        return x;
    };
    for (int q = tid; q < 64 * (K1 / 8); q += 128 * DR_GROUPS) {
        const int n = q / (K1 / 8), j = q % (K1 / 8);
        if (j < 4) {
            float v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = wv(p.w.w1[n * 32 + 8 * j + e]);
            put8(sm + DRO_W1, n, j, K1, v);
        } else if (j == 4) put_bias_chunk(sm + DRO_W1, n, j, K1, bv(p.w.b1[n]), false);
        else put_zero_chunk(sm + DRO_W1, n, j, K1);
    }
    for (int q = tid; q < 64 * (K2 / 8); q += 128 * DR_GROUPS) {
        const int n = q / (K2 / 8), j = q % (K2 / 8);
        if (j < 8) {
            float v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = wv(p.w.w2[n * 64 + 8 * j + e]);
            put8(sm + DRO_W2, n, j, K2, v);
        } else if (j == 8) put_bias_chunk(sm + DRO_W2, n, j, K2, bv(p.w.b2[n]), false);
        else put_zero_chunk(sm + DRO_W2, n, j, K2);
    }
    for (int q = tid; q < DR_NC * (K2 / 8); q += 128 * DR_GROUPS) {
        const int n = q / (K2 / 8), j = q % (K2 / 8);
        if (n >= nc || j == 9) put_zero_chunk(sm + DRO_W3, n, j, K2);
        else if (j < 8) {
            float v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = wv(p.w.w3[n * 64 + 8 * j + e]);
            put8(sm + DRO_W3, n, j, K2, v);
        } else put_bias_chunk(sm + DRO_W3, n, j, K2, bv(p.w.b3[n]), false);
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = s_tmem + (uint32_t)DR_COLS * (uint32_t)group;
    const uint32_t my_lane = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    unsigned char *ga = sm + DRO_A + group * DR_GROUP_BYTES;
    float *rows_tile = reinterpret_cast<float *>(sm + DRO_ROWS) + warp * 32 * 33;
    const uint32_t sa_a = ptx::smem_u32(ga), sa_w1 = ptx::smem_u32(sm + DRO_W1), sa_w2 = ptx::smem_u32(sm + DRO_W2),
                   sa_w3 = ptx::smem_u32(sm + DRO_W3);
    uint32_t phase = 0;
    __half2 hmax = __float2half2_rn(0.0f);
    bool first_wait = p.test_timeout != 0;
    auto issue_layer = [&](uint32_t b_addr, int K, int N) {
        if (m == 0) {
            fence_after();
            gemm(tmem, sa_a, b_addr, K, N);
            mma_commit(&s_bar[group]);
        }
    };
    auto wait_layer = [&]() -> bool {
        const bool ok = first_wait ? ptx::mbar_wait_bounded(&s_never, 0, TEST_WAIT_LIMIT_NS)
                                   : ptx::mbar_wait_bounded(&s_bar[group], phase, LT_WAIT_NS);
        first_wait = false;
        if (!ok) s_fail[group] = 1;
        group_sync(group);
        fence_after();
        if (s_fail[group]) return false;
        phase ^= 1u;
        return true;
    };
    auto run_layer = [&](uint32_t b_addr, int K, int N) -> bool {
        issue_layer(b_addr, K, N);
        return wait_layer();
    };
    auto hand_off = [&]() {
        fence_async_smem();
        fence_before();
        group_sync(group);
    };
    const uint32_t n_tiles = (p.n + 127) / 128;
    const uint32_t first = blockIdx.x * DR_GROUPS + group, step = gridDim.x * DR_GROUPS;
    // this thread's row of a tile: the gathered FP32 latent (all zero past the end)
    auto gather = [&](uint32_t tile, float x[32]) {
        const uint32_t rec = tile * 128 + (uint32_t)m;
        const bool ok = tile < n_tiles && rec < p.n;
        const size_t src = ok ? p.perm[rec] : 0;
        warp_load_rows<32>(x, p.latents, src * 32, ok, 0, 32, rows_tile);
    };
    float xn[32];
    gather(first, xn);
    for (uint32_t tile = first; tile < n_tiles; tile += step) {
        const uint32_t rec = tile * 128 + (uint32_t)m;
        const bool valid = rec < p.n;
        {
            __half2 hx = __float2half2_rn(0.0f);
#pragma unroll
            for (int j = 0; j < 4; ++j) {  // FP16 latents, as the inference decoder holds them
                put8(ga, m, j, K1, xn + 8 * j);
#pragma unroll
                for (int e = 0; e < 8; ++e) hx = __hmax2(hx, __float2half2_rn(fabsf(xn[8 * j + e])));
            }
            hmax = __hmax2(hmax, hx);
            put_bias_chunk(ga, m, 4, K1, 0.0f, true);
            put_zero_chunk(ga, m, 5, K1);
        }
        hand_off();
        if (!run_layer(sa_w1, K1, 64)) break;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float v[32];
            tmem_ld32(my_lane + 32 * h, v);
#pragma unroll
            for (int c = 0; c < 4; ++c) put8_relu(ga, m, 4 * h + c, K2, v + 8 * c, hmax);
        }
        put_bias_chunk(ga, m, 8, K2, 0.0f, true);
        put_zero_chunk(ga, m, 9, K2);
        hand_off();
        if (!run_layer(sa_w2, K2, 64)) break;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float v[32];
            tmem_ld32(my_lane + 32 * h, v);
#pragma unroll
            for (int c = 0; c < 4; ++c) put8_relu(ga, m, 4 * h + c, K2, v + 8 * c, hmax);
        }
        hand_off();
        // Y -> record `rec` in two halves: columns < n1 to the density record,
        // the rest to the SH record; the next tile's latents are gathered
        // while the first half's MMAs run
        bool ok = true;
#pragma unroll 1
        for (int half = 0; half < 2 && ok; ++half) {
            const int n_cols = half ? DR_NH1 : DR_NH0, col0 = half ? DR_NH0 : 0;
            issue_layer(sa_w3 + (uint32_t)core_off(col0, 0, K2), K2, n_cols);
            if (half == 0) gather(tile + step, xn);
            if (!(ok = wait_layer())) break;
#pragma unroll 1
            for (int c = 0; c < DR_NH0 / 32; ++c) {
                float v[32];
                tmem_ld32(my_lane + 32 * c, v);  // columns past n_cols: the group's unused scratch
                warp_store_rows<32>(v, p.sig, (size_t)rec * p.ss, p.zc, (size_t)rec * p.zs, p.n1, valid,
                                    col0 + 32 * c, col0 + n_cols < nc ? col0 + n_cols : nc, rows_tile);
            }
            fence_before();  // TMEM reads done before the group's next MMAs
            group_sync(group);
        }
        if (!ok) break;
    }
    if (p.status && (!(__low2float(hmax) <= F16_MAX) || !(__high2float(hmax) <= F16_MAX) || (tid == 0 && s_range)))
        atomicOr(p.status, STATUS_FP16_RANGE);
    if (s_fail[group] && m == 0) {
        ptx::mbar_wait_bounded(&s_bar[group], phase, LT_WAIT_NS);
        if (p.status) atomicOr(p.status, STATUS_DEVICE_TIMEOUT);
    }
    __syncthreads();
    fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_tmem), "r"(512u) : "memory");
}

// cuTensorMapEncodeTiled from the driver, looked up once.
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }();
    return fn;
}

int launch_latent_table(const LatentParams &pin, int sm_count, void *stream)
{
    if (pin.n_leaves == 0) return (int)cudaSuccess;
    LatentParams p = pin;
    // the table as a 2-D tensor [n_leaves][32] of FP32 (128-byte rows) or FP16
    // (64-byte rows), stored in boxes of 128 rows from swizzled shared memory
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return (int)cudaErrorNotSupported;
    const cuuint64_t dims[2] = {TABLE_STRIDE, p.n_leaves};
    const cuuint64_t strides[1] = {TABLE_STRIDE * (p.half_table ? 2u : 4u)};
    const cuuint32_t box[2] = {TABLE_STRIDE, LT_M};
    const cuuint32_t estr[2] = {1, 1};
    if (enc(&p.table_map, p.half_table ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
            p.table, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            p.half_table ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return (int)cudaErrorInvalidValue;
    auto launch = [&](auto kern, int G, int smem, int ctas_per_sm) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     p.carveout > 0 ? p.carveout : (int)cudaSharedmemCarveoutDefault);
        if (e != cudaSuccess) return e;
        int per_sm = ctas_per_sm;
        if (per_sm <= 0) {
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128 * G, smem);
            if (e != cudaSuccess) return e;
            if (per_sm < 1) per_sm = 1;
        }
        if (per_sm * 64 * G > 512) per_sm = 512 / (64 * G);  // TMEM has 512 columns
        const uint32_t n_tiles = (p.n_leaves + LT_M - 1) / LT_M;
        uint64_t blocks = (uint64_t)sm_count * per_sm;
        const uint64_t need = (n_tiles + G - 1) / G;
        if (blocks > need) blocks = need;
        kern<<<(unsigned)blocks, 128 * G, smem, (cudaStream_t)stream>>>(p);
        return cudaGetLastError();
    };
    if (p.pipeline)
        return (int)launch(latent_table_kernel<LT_GROUPS_PIPE>, LT_GROUPS_PIPE, lt_smem<LT_GROUPS_PIPE>(), 1);
    return (int)launch(latent_table_kernel<LT_GROUPS_FULL>, LT_GROUPS_FULL, lt_smem<LT_GROUPS_FULL>(), 0);
}

int latent_pipeline_smem_bytes() { return lt_smem<LT_GROUPS_PIPE>(); }

int launch_decode_records_tc(const fpo_mlp &w, int n1, int n2, uint32_t n, const float *latents, const uint32_t *perm,
                             float *sig, float *zc, uint32_t *status, bool test_timeout, int sm_count, void *stream)
{
    if (n == 0) return (int)cudaSuccess;
    DecodeTcParams p{};
    p.w = w;
    p.latents = latents;
    p.perm = perm;
    p.sig = sig;
    p.zc = zc;
    p.n = n;
    p.n1 = n1;
    p.nc = n1 + 27 * n2;
    p.ss = sig_stride(n1);
    p.zs = z_stride(n2);
    p.status = status;
    p.test_timeout = test_timeout;
    const int smem = DR_SMEM + 1024;
    cudaError_t e = cudaFuncSetAttribute(decode_records_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return (int)e;
    const uint32_t n_tiles = (n + 127) / 128;
    const uint32_t need = (n_tiles + DR_GROUPS - 1) / DR_GROUPS;
    const uint32_t blocks = need < (uint32_t)sm_count ? need : (uint32_t)sm_count;
    decode_records_tc_kernel<<<blocks, 128 * DR_GROUPS, smem, (cudaStream_t)stream>>>(p);
    return (int)cudaGetLastError();
}

}  // namespace fpo

extern "C" int fpo_decoder_grad_tc(const fpo_mlp *w, int32_t n1, int32_t n2, uint32_t batch, const uint32_t *rows,
                                   const float *latents, const float *targets, const float *coef_weight,
                                   const float *extra_dy, const fpo_mlp *grad, float *dlatents, double *loss,
                                   uint32_t *status, uint32_t flags, void *cuda_stream)
{
    using namespace fpo;
    if (!w || !grad || !w->w1 || !w->b1 || !w->w2 || !w->b2 || !w->w3 || !w->b3 || !grad->w1 || !grad->b1 ||
        !grad->w2 || !grad->b2 || !grad->w3 || !grad->b3)
        return set_last_error(FPO_ERR_INVALID_ARG, "NULL weights");
    if (n1 < 1 || n2 < 1 || n1 + 27 * n2 > TG_NC) return set_last_error(FPO_ERR_INVALID_ARG, "n1 + 27 n2 must be in [28, 176]");
    if (flags & ~(uint32_t)FPO_FLAG_TEST_DEVICE_TIMEOUT) return set_last_error(FPO_ERR_INVALID_ARG, "unknown flags");
    if (batch == 0) return FPO_OK;
    if (!rows || !latents || !targets || !coef_weight || !dlatents) return set_last_error(FPO_ERR_INVALID_ARG, "NULL array");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return set_last_error(FPO_ERR_CUDA, cudaGetErrorString(e));
    DecoderGradTcParams p{};
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
    p.status = status;
    p.nc = n1 + 27 * n2;
    p.test_timeout = (flags & FPO_FLAG_TEST_DEVICE_TIMEOUT) != 0;
    const int smem = TG_SMEM;
    e = cudaFuncSetAttribute(decoder_grad_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return set_last_error(FPO_ERR_CUDA, cudaGetErrorString(e));
    const uint32_t n_tiles = (batch + 127) / 128;
    const uint32_t blocks = n_tiles < (uint32_t)sms ? n_tiles : (uint32_t)sms;
    decoder_grad_tc_kernel<<<blocks, 128, smem, (cudaStream_t)cuda_stream>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_last_error(FPO_ERR_CUDA, cudaGetErrorString(e));
    return FPO_OK;
}

using namespace fpo;

extern "C" int fpo_latent_table(const fpo_decoder *dec, int32_t n1, int32_t n2, double t, double period_T,
                                uint32_t n_leaves, const uint16_t *latents, float *table, uint32_t *status,
                                void *cuda_stream)
{
    if (!dec) return set_last_error(FPO_ERR_INVALID_ARG, "dec is NULL");
    if (n1 < 1 || n1 > 32 || n2 < 1 || n2 > 16) return set_last_error(FPO_ERR_INVALID_ARG, "n1 in [1, 32], n2 in [1, 16]");
    if (!(period_T > 0.0)) return set_last_error(FPO_ERR_INVALID_ARG, "period_T must be > 0");
    if (n_leaves == 0) return FPO_OK;
    if (!latents || !table || !dec->w1 || !dec->b1 || !dec->w2 || !dec->b2 || !dec->w3 || !dec->b3)
        return set_last_error(FPO_ERR_INVALID_ARG, "NULL array");
    if (reinterpret_cast<uintptr_t>(latents) % 16 != 0 || reinterpret_cast<uintptr_t>(table) % 16 != 0)
        return set_last_error(FPO_ERR_INVALID_ARG, "latents and table must be 16-byte aligned");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return set_last_error(FPO_ERR_CUDA, cudaGetErrorString(e));
    LatentParams p{};
    p.latents = latents;
    p.w1 = dec->w1;
    p.b1 = dec->b1;
    p.w2 = dec->w2;
    p.b2 = dec->b2;
    p.w3 = dec->w3;
    p.b3 = dec->b3;
    p.n1 = n1;
    p.n2 = n2;
    p.t = t;
    p.period_T = period_T;
    p.n_leaves = n_leaves;
    p.table = table;
    p.status = status;
    const int ce = launch_latent_table(p, sms, cuda_stream);
    if (ce != cudaSuccess) return set_last_error(FPO_ERR_CUDA, cudaGetErrorString((cudaError_t)ce));
    return FPO_OK;
}
