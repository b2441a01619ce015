// sg.cu -- surrogate hardness model: message-passing network over the Chimera
// coupler graph that predicts log10 TTS (C ABI: sg_* in include/pt.h).
//
// The paper has no surrogate; it is this library's way to spend PT evaluations
// (Sec. II TTS inside Algorithm 1) only on promising coupler moves.  Network:
//   h0_i = X[u_i], e0_e = Jt[idx(J_e)]                      (u: orientation)
//   per layer: m_i = sum_{j in N(i)} relu(Wm [h_j, e_ij] + bm)
//              h_i += relu(Wu [h_i, m_i] + bu)
//              e_ij += relu(We [e_ij, h_i + h_j] + be)        (updated h)
//   readout:   y = w2 . relu(W1 mean_i(h_i) + b1) + b2
// Hidden width 64.  Weights and activations are BF16, accumulation FP32; the
// three per-layer linear maps (K = 128 -> 64 outputs over every message,
// node or edge row), their input gradients and their weight gradients run on
// the 5th-generation tensor cores (tcgen05.mma, accumulators in tensor
// memory).  Gradients are FP32 buffers; master weights and Adam moments are
// FP32.  Every reduction runs in a fixed order (no floating-point atomics), so
// a training step is bit-reproducible.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/pt.h"
#include "pt_internal.h"

namespace {

constexpr int HD = 64;      // hidden width
constexpr int KIN = 128;    // input width of every linear map: [64 | 64]
constexpr int MAXDEG = 6;
typedef __nv_bfloat16 bf16;

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ uint32_t pack_bf2(float a, float b)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ float2 unpack_bf2(uint32_t u)
{
    __nv_bfloat162 v = *reinterpret_cast<__nv_bfloat162*>(&u);
    return __bfloat1622float2(v);
}

// Row r of a linear map's input is [P0[idx0(r)] | P1[idx1(r)]] with
// idx(r) = (r / R_local) * S + map[r % R_local] (64 BF16 per row each).
struct RowSrc {
    const bf16* P0;
    const int* map0;
    int S0;
    const bf16* P1;
    const int* map1;
    int S1;
    int R_local;
    __device__ __forceinline__ const uint32_t* half(int r, int which) const
    {
        const int b = r / R_local, l = r - b * R_local;
        if (which == 0) return reinterpret_cast<const uint32_t*>(P0 + ((size_t)b * S0 + map0[l]) * HD);
        return reinterpret_cast<const uint32_t*>(P1 + ((size_t)b * S1 + map1[l]) * HD);
    }
};

// Floats of one CTA's weight-gradient partial: dW [64][128] then db [64].
constexpr int WPART = HD * KIN + HD;

// dW += sum over blocks of the partials (and db likewise), in a fixed order:
// stage 1 (grid.y = WRED_GROUPS) sums consecutive ranges of the partials
// into `tmp`, stage 2 adds the group sums in order.
constexpr int WRED_GROUPS = 16;
__global__ void lin_wgrad_reduce1(int nblocks, const float* __restrict__ part, float* __restrict__ tmp)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= WPART) return;
    const int per = (nblocks + WRED_GROUPS - 1) / WRED_GROUPS;
    const int b0 = blockIdx.y * per, b1 = min(nblocks, b0 + per);
    float s0 = 0.f, s1 = 0.f;
    int b = b0;
    for (; b + 2 <= b1; b += 2) {
        s0 += part[(size_t)b * WPART + i];
        s1 += part[(size_t)(b + 1) * WPART + i];
    }
    if (b < b1) s0 += part[(size_t)b * WPART + i];
    tmp[(size_t)blockIdx.y * WPART + i] = s0 + s1;
}

__global__ void lin_wgrad_reduce2(const float* __restrict__ tmp, float* __restrict__ dW, float* __restrict__ db)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= WPART) return;
    float s = 0.f;
    for (int g = 0; g < WRED_GROUPS; ++g) s += tmp[(size_t)g * WPART + i];
    if (i < HD * KIN) dW[i] += s;
    else db[i - HD * KIN] += s;
}

// ------------------------------------------- tcgen05 (5th-generation tensor core) GEMMs
// The forward maps Z = X W^T + b (128 rows x K = 128 -> 64 outputs per tile)
// and the input gradient dX = dZ W (128 rows x K = 64 -> 128 inputs per
// tile) run on tcgen05.mma with the accumulator in tensor memory:
//   * one CTA of 128 threads per 128-row tile (persistent over tiles); one
//     thread issues the MMAs and commits them to an mbarrier;
//   * operands in shared memory in the canonical K-major layout without
//     swizzle, built from 8-row x 16-byte core matrices stored as
//     [8-row group][k-chunk of 8 elements][8 rows][16 bytes]: core matrices
//     adjacent in K are 128 bytes apart (the leading byte offset) and 8-row
//     groups (number of k-chunks) x 128 bytes apart (the stride byte offset).
//     Read with the two offsets the other way round, every address would
//     still lie inside the 48 KB the kernels allocate;
//   * the weights, pre-packed in that layout (pack_weights_kernel), arrive by
//     one bulk asynchronous copy; the gathered input rows by 16-byte cp.async;
//   * after the commit each warp reads its 32 accumulator rows (TMEM lanes
//     32w .. 32w+31) with tcgen05.ld, one row per thread, for the epilogue;
//   * every mbarrier wait is bounded: on a timeout the CTA records it in
//     *err, stops taking tiles, frees its tensor memory and returns.
constexpr uint32_t TC_WAIT_LIMIT = 1u << 22;
constexpr int TC_ROWS = 128;
// CTAs of 256 threads: all 8 warps stage a tile; in the epilogue warps w and
// w + 4 read the same 32 tensor-memory lanes (a warp reaches lanes
// 32 (w mod 4) .. + 31) and split the columns, and each warp's stores pass
// through a 4 KB slice of the consumed operand buffer (warp_store_*).
// Dynamic shared memory: forward A 32 KB + W 16 KB = 48 KB, input gradient
// dZ 16 KB + staging 16 KB + W^T 16 KB = 48 KB (4 CTAs per SM, 64 or 128
// tensor-memory columns each);
// weight gradient two stages of 24 KB (the next chunk loads while the
// current one is multiplied) + ones 16 KB = 64 KB (3 CTAs, 128 columns).  The
// shared memory bounds the resident CTAs, so their tensor memory never
// exceeds an SM's 512 columns; the persistent grids use exactly that many.
constexpr int TC_THREADS = 256;
constexpr int TC_A_FWD = TC_ROWS * KIN * 2, TC_A_BWD = TC_ROWS * HD * 2;
constexpr int TC_SMEM_FWD = TC_A_FWD + HD * KIN * 2;
constexpr int TC_SMEM_BWD = TC_SMEM_FWD;
constexpr int TC_CTAS_FWD = 4, TC_CTAS_BWD = 4, TC_CTAS_WGRAD = 3;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of tcgen05.mma: start address, leading and
// stride byte offsets (all >> 4), descriptor version 1 (bits 46-47), no
// swizzle (layout type 0 in bits 61-63), base offset 0.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor, kind::f16: F32 accumulator (bits 4-5 = 1), BF16 A
// and B (bits 7-9, 10-12 = 1), both K-major, N >> 3 in bits 17-22, M >> 4 in
// bits 24-28.
__host__ __device__ constexpr uint32_t tc_idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity)
{
    for (uint32_t i = 0; i < TC_WAIT_LIMIT; ++i) {
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(smem_u32(bar)), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}

// One bulk asynchronous copy global -> shared of `bytes` (a multiple of 16,
// both addresses 16-byte aligned), completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accum)
{
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                 ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
                 : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Epilogue stores of one warp's 32 accumulator rows (lane l holds row l),
// staged through a 4 KB slice of shared memory so that each global store
// instruction writes whole rows: 4 rows x 128 bytes (32 FP32 columns) or 8
// rows x 64 bytes (32 BF16 columns) instead of one 16-byte piece of each of
// 32 rows.  Row l's 16-byte chunk c sits at slot c ^ (l & 7) (FP32) or
// c ^ ((l >> 1) & 3) (BF16) of its row, so neither the row-wise writes nor
// the chunk-wise reads of a warp meet a bank conflict.  flush_* writes the
// staged block: g points at the warp's first row and first column, ld is the
// row pitch in elements, and only rows < nvalid are written.
__device__ __forceinline__ void stage_f32(unsigned char* stage, int lane, int c, float4 v)
{
    *reinterpret_cast<float4*>(stage + lane * 128 + ((c ^ (lane & 7)) << 4)) = v;
}

__device__ __forceinline__ void flush_f32x32(const unsigned char* stage, float* g, int ld, int nvalid, int lane)
{
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int row = k * 4 + (lane >> 3), c = lane & 7;
        const float4 x = *reinterpret_cast<const float4*>(stage + row * 128 + ((c ^ (row & 7)) << 4));
        if (row < nvalid) *reinterpret_cast<float4*>(g + (size_t)row * ld + c * 4) = x;
    }
    __syncwarp();
}

// Adds the sums of staged row pairs (2p, 2p + 1), in that order, to row p of g
// (16 pairs x 32 FP32 columns; only pairs < npairs).
__device__ __forceinline__ void flush_pairs_add_f32x32(const unsigned char* stage, float* g, int ld, int npairs,
                                                       int lane)
{
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int p = k * 4 + (lane >> 3), c = lane & 7, ra = 2 * p, rb = ra + 1;
        const float4 a = *reinterpret_cast<const float4*>(stage + ra * 128 + ((c ^ (ra & 7)) << 4));
        const float4 b = *reinterpret_cast<const float4*>(stage + rb * 128 + ((c ^ (rb & 7)) << 4));
        if (p < npairs) {
            float4* gp = reinterpret_cast<float4*>(g + (size_t)p * ld + c * 4);
            float4 o = *gp;
            o.x += a.x + b.x;
            o.y += a.y + b.y;
            o.z += a.z + b.z;
            o.w += a.w + b.w;
            *gp = o;
        }
    }
    __syncwarp();
}

__device__ __forceinline__ void stage_bf16(unsigned char* stage, int lane, int c, uint4 v)
{
    *reinterpret_cast<uint4*>(stage + lane * 64 + ((c ^ ((lane >> 1) & 3)) << 4)) = v;
}

__device__ __forceinline__ void flush_bf16x32(const unsigned char* stage, bf16* g, int ld, int nvalid, int lane)
{
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int row = k * 8 + (lane >> 2), c = lane & 3;
        const uint4 x = *reinterpret_cast<const uint4*>(stage + row * 64 + ((c ^ ((row >> 1) & 3)) << 4));
        if (row < nvalid) *reinterpret_cast<uint4*>(g + (size_t)row * ld + c * 8) = x;
    }
    __syncwarp();
}

// A 32-column BF16 block packed in 16 words (2 per column pair) through the staging slice.
__device__ __forceinline__ void store_bf16x32(unsigned char* stage, const uint32_t (&w)[16], bf16* g, int ld,
                                              int nvalid, int lane)
{
#pragma unroll
    for (int c = 0; c < 4; ++c) stage_bf16(stage, lane, c, make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]));
    flush_bf16x32(stage, g, ld, nvalid, lane);
}

// Common prologue: tensor memory (ncols columns, warp 0), the two mbarriers,
// and the packed weights (bytes) by one bulk copy.  Returns false (for every
// thread) if the weights did not arrive within the wait limit.
__device__ __forceinline__ bool tc_setup(uint32_t* tmem_sh, uint64_t* bar_w, uint64_t* bar_mma, uint32_t ncols,
                                         void* Ws, const void* Wpk, uint32_t bytes)
{
    const int tid = threadIdx.x;
    if ((tid >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_sh)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(bar_w, 1);
        mbar_init(bar_mma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (bytes == 0) return true;
    if (tid == 0) bulk_g2s(Ws, Wpk, bytes, bar_w);
    bool ok = mbar_wait(bar_w, 0);
    if (!ok) ok = mbar_wait(bar_w, 0);         // second bounded wait for the copy still in flight
    return !__syncthreads_or(!ok);
}

__device__ __forceinline__ void tc_teardown(uint32_t tmem, uint32_t ncols, bool failed, int* err)
{
    tc_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    }
    if (failed && threadIdx.x == 0) atomicExch(err, 1);
}

// Forward: Z = X W^T + bias over `rows` gathered rows (see RowSrc).  EPI 0
// (messages): Z -> Zout (BF16), relu(Z) -> Rout (FP32).  EPI 1 (residual):
// Z -> Zout, Yout = P0 row + relu(Z) (BF16).
template <int EPI>
__global__ void __launch_bounds__(TC_THREADS, TC_CTAS_FWD) lin_fwd_tc_kernel(int rows, RowSrc src, const bf16* __restrict__ Wpk,
                                                                const float* __restrict__ bias, bf16* __restrict__ Zout,
                                                                float* __restrict__ Rout, bf16* __restrict__ Yout,
                                                                int* err)
{
    extern __shared__ __align__(128) unsigned char tc_smem[];
    unsigned char* As = tc_smem;                         // [16 row groups][16 k-chunks][8 rows][16 B]
    unsigned char* Ws = tc_smem + TC_A_FWD;              // [8 output groups][16 k-chunks][8 outputs][16 B]
    __shared__ __align__(8) uint64_t bar_w, bar_mma;
    __shared__ uint32_t tmem_sh;
    __shared__ const unsigned char* rowp[2][2][TC_ROWS]; // gathered row halves of this and the next tile (NULL past the end)
    __shared__ float bias_sm[HD];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid < HD) bias_sm[tid] = bias[tid];
    bool failed = !tc_setup(&tmem_sh, &bar_w, &bar_mma, 64, Ws, Wpk, HD * KIN * 2);
    const uint32_t tmem = tmem_sh;
    constexpr uint32_t IDESC = tc_idesc_bf16(TC_ROWS, HD);
    const int ntiles = (rows + TC_ROWS - 1) / TC_ROWS;
    uint32_t phase = 0;
    // one index lookup per row half: thread tid looks up row tid mod 128, half tid / 128
    auto lookup = [&](int t, int buf) {
        const int row = tid & (TC_ROWS - 1), hf = tid >> 7, r = t * TC_ROWS + row;
        rowp[buf][hf][row] = r < rows ? reinterpret_cast<const unsigned char*>(src.half(r, hf)) : nullptr;
    };
    if (blockIdx.x < ntiles) lookup(blockIdx.x, 0);
    int buf = 0;
    for (int tile = blockIdx.x; !failed && tile < ntiles; tile += gridDim.x, buf ^= 1) {
        const int r0 = tile * TC_ROWS;
        __syncthreads();                                    // this tile's row pointers staged; the last epilogue done
        for (int i = tid; i < 16 * TC_ROWS; i += TC_THREADS) {   // chunk i: row (i >> 7) * 8 + (i & 7), k-chunk (i >> 3) & 15
            const int kc = (i >> 3) & 15, row = ((i >> 7) << 3) | (i & 7);
            const unsigned char* p = rowp[buf][kc >> 3][row];
            cp_async16(As + i * 16, p ? p + (kc & 7) * 16 : reinterpret_cast<const unsigned char*>(Wpk), p != nullptr);
        }
        // the next tile's lookups overlap this gather (its buffer was last read by the previous gather)
        if (tile + (int)gridDim.x < ntiles) lookup(tile + gridDim.x, buf ^ 1);
        asm volatile("cp.async.wait_all;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");     // visible to the tensor core
        tc_fence_before();
        __syncthreads();                                    // also: the previous tile's TMEM reads are done
        tc_fence_after();
        if (tid == 0) {
#pragma unroll
            for (int ks = 0; ks < KIN / 16; ++ks)
                tc_mma(tmem, tc_desc(smem_u32(As) + ks * 256, 128, 16 * 128), tc_desc(smem_u32(Ws) + ks * 256, 128, 16 * 128),
                       IDESC, ks > 0 ? 1u : 0u);
            tc_commit(&bar_mma);
        }
        const bool ok = mbar_wait(&bar_mma, phase);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        tc_fence_after();
        // warp w: accumulator rows 32 (w mod 4) .. + 31 (TMEM lanes), columns 32 (w / 4) .. + 31, read
        // 16 at a time; the operand tile is consumed (MMA complete), so its 32 KB hold the 8 warps'
        // staging slices
        const int q = warp & 3, cb = (warp >> 2) * (HD / 2), row0 = r0 + q * 32, row = q * 32 + lane;
        const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16);
        unsigned char* stage = As + warp * 4096;
        uint32_t zw[HD / 4], yw[EPI == 1 ? HD / 4 : 1];
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            const int c0 = cb + 16 * hh;
            float z[16];
            tmem_ld16(tl + c0, z);
            tmem_ld_wait();
#pragma unroll
            for (int i = 0; i < 16; ++i) z[i] += bias_sm[c0 + i];
#pragma unroll
            for (int i = 0; i < 8; ++i) zw[8 * hh + i] = pack_bf2(z[2 * i], z[2 * i + 1]);
            if (EPI == 0) {
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    stage_f32(stage, lane, 4 * hh + c,
                              make_float4(fmaxf(z[4 * c], 0.f), fmaxf(z[4 * c + 1], 0.f), fmaxf(z[4 * c + 2], 0.f),
                                          fmaxf(z[4 * c + 3], 0.f)));
            } else {
                // the residual input is half 0 of this row, already staged: k-chunks c0/8 and c0/8 + 1
#pragma unroll
                for (int kc = 0; kc < 2; ++kc) {
                    const uint4 b4 = *reinterpret_cast<const uint4*>(As + (((row >> 3) * 16 + (c0 >> 3) + kc) * 128) +
                                                                     (row & 7) * 16);
                    const uint32_t bw[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float2 bb = unpack_bf2(bw[i]);
                        yw[(EPI == 1 ? 8 * hh + 4 * kc + i : 0)] =
                            pack_bf2(bb.x + fmaxf(z[8 * kc + 2 * i], 0.f), bb.y + fmaxf(z[8 * kc + 2 * i + 1], 0.f));
                    }
                }
            }
        }
        if constexpr (EPI == 0) {
            flush_f32x32(stage, Rout + (size_t)row0 * HD + cb, HD, rows - row0, lane);
        } else {
            __syncthreads();                               // every residual read before any slice is overwritten
            store_bf16x32(stage, yw, Yout + (size_t)row0 * HD + cb, HD, rows - row0, lane);
        }
        store_bf16x32(stage, zw, Zout + (size_t)row0 * HD + cb, HD, rows - row0, lane);
    }
    tc_teardown(tmem, 64, failed, err);
}

// Input gradient: dX = dZ W over `rows` rows of dZ [rows][64] (BF16), with
// W^T pre-packed.  EPI 0 (messages; rows 2e and 2e+1 are the two directions
// of edge e): dX[:, :64] -> dX [rows][64] FP32, and the edge half of each
// pair, dX[2e][64:] + dX[2e+1][64:], added to out1[e] ([rows / 2][64]).
// EPI 1 (node and edge updates): out0 = base + dX[:, :64] (base may be out0
// or NULL) and out1 = dX[:, 64:], both [rows][64] FP32.
template <int EPI>
__global__ void __launch_bounds__(TC_THREADS, EPI == 0 ? TC_CTAS_BWD : 2) lin_bwd_input_tc_kernel(int rows, const bf16* __restrict__ dZ,
                                                                      const bf16* __restrict__ WTpk,
                                                                      float* __restrict__ dX, const float* base,
                                                                      float* out0, float* __restrict__ out1, int* err)
{
    extern __shared__ __align__(128) unsigned char tc_smem[];
    unsigned char* As = tc_smem;                         // [16 row groups][8 k-chunks][8 rows][16 B]
    unsigned char* Ws = tc_smem + 2 * TC_A_BWD;          // [16 input groups][8 k-chunks][8 inputs][16 B]
    // bytes [0, 2 * TC_A_BWD): the dZ tile, then (MMA complete) the epilogue's staging slices
    __shared__ __align__(8) uint64_t bar_w, bar_mma;
    __shared__ uint32_t tmem_sh;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    bool failed = !tc_setup(&tmem_sh, &bar_w, &bar_mma, 128, Ws, WTpk, KIN * HD * 2);
    const uint32_t tmem = tmem_sh;
    constexpr uint32_t IDESC = tc_idesc_bf16(TC_ROWS, KIN);
    const int ntiles = (rows + TC_ROWS - 1) / TC_ROWS;
    uint32_t phase = 0;
    for (int tile = blockIdx.x; !failed && tile < ntiles; tile += gridDim.x) {
        const int r0 = tile * TC_ROWS;
        for (int i = tid; i < 8 * TC_ROWS; i += TC_THREADS) {    // chunk i: row (i >> 6) * 8 + (i & 7), k-chunk (i >> 3) & 7
            const int kc = (i >> 3) & 7, row = ((i >> 6) << 3) | (i & 7), r = r0 + row;
            const bool v = r < rows;
            const unsigned char* g = v ? reinterpret_cast<const unsigned char*>(dZ + (size_t)r * HD) + kc * 16
                                       : reinterpret_cast<const unsigned char*>(WTpk);
            cp_async16(As + i * 16, g, v);
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
#pragma unroll
            for (int ks = 0; ks < HD / 16; ++ks)
                tc_mma(tmem, tc_desc(smem_u32(As) + ks * 256, 128, 8 * 128), tc_desc(smem_u32(Ws) + ks * 256, 128, 8 * 128),
                       IDESC, ks > 0 ? 1u : 0u);
            tc_commit(&bar_mma);
        }
        const int q = warp & 3, r = r0 + q * 32 + lane;
        // warps 0-3 add this row's base gradient to dX[:, :64]: loaded while the MMAs run
        float4 bpre[EPI == 1 ? HD / 4 : 1];
        if (EPI == 1 && warp < 4 && base && r < rows) {
#pragma unroll
            for (int i = 0; i < HD / 4; ++i) bpre[i] = reinterpret_cast<const float4*>(base + (size_t)r * HD)[i];
        } else {
#pragma unroll
            for (int i = 0; i < (EPI == 1 ? HD / 4 : 1); ++i) bpre[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const bool ok = mbar_wait(&bar_mma, phase);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        tc_fence_after();
        // warp w: rows 32 (w mod 4) .. + 31, columns 64 (w / 4) .. + 63 of dX, in two passes of 32
        // through its staging slice (the consumed dZ tile and the 16 KB above it)
        const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16);
        const int row0 = r0 + q * 32;
        unsigned char* stage = As + warp * 4096;
#pragma unroll
        for (int pass = 0; pass < 2; ++pass) {
            const int c0 = (warp >> 2) * HD + pass * 32;
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                float d[16];
                tmem_ld16(tl + c0 + 16 * hh, d);
                tmem_ld_wait();
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    float4 v = make_float4(d[4 * c], d[4 * c + 1], d[4 * c + 2], d[4 * c + 3]);
                    if (EPI == 1 && c0 < HD) {
                        const float4 bb = bpre[(EPI == 1 ? (c0 >> 2) + 4 * hh + c : 0)];
                        v.x += bb.x;
                        v.y += bb.y;
                        v.z += bb.z;
                        v.w += bb.w;
                    }
                    stage_f32(stage, lane, 4 * hh + c, v);
                }
            }
            if (EPI == 0 && c0 < HD)
                flush_f32x32(stage, dX + (size_t)row0 * HD + c0, HD, rows - row0, lane);
            else if (EPI == 0)                             // a warp's 32 rows are 16 whole edges (row0 is even)
                flush_pairs_add_f32x32(stage, out1 + (size_t)(row0 / 2) * HD + (c0 - HD), HD, (rows - row0) / 2, lane);
            else if (c0 < HD)
                flush_f32x32(stage, out0 + (size_t)row0 * HD + c0, HD, rows - row0, lane);
            else
                flush_f32x32(stage, out1 + (size_t)row0 * HD + (c0 - HD), HD, rows - row0, lane);
        }
        __syncthreads();                                   // staging slices read before the next tile lands there
    }
    tc_teardown(tmem, 128, failed, err);
}

// Weight gradient: dW = dZ^T X and db = column sums of dZ over `rows` rows,
// as D[in][o] = sum_r X[r][in] dZ[r][o] (M = 128 inputs, N = 64 outputs,
// K = rows) accumulated in tensor memory over the CTA's 64-row chunks c =
// blockIdx.x, c += gridDim.x; db the same with a tile of ones in place of X.
// Both operands are MN-major: a 16-byte chunk of a row of X (8 inputs) or of
// dZ (8 outputs) is one row of a core matrix, so the rows are staged with
// 16-byte cp.async and no transposition, as [MN group][k group][8 rows][16 B].
// Each CTA writes its partial [64][128] + [64] like lin_wgrad_kernel, and
// lin_wgrad_reduce1/2 add the partials in a fixed order.
constexpr int TC_WCH = 64;                          // rows per chunk
constexpr int TC_WSTAGE = TC_WCH * KIN * 2 + TC_WCH * HD * 2;          // X 16 KB + dZ 8 KB
constexpr int TC_SMEM_WGRAD = 2 * TC_WSTAGE + TC_WCH * KIN * 2;         // two stages + ones 16 KB
__global__ void __launch_bounds__(TC_THREADS) lin_wgrad_tc_kernel(int rows, const bf16* __restrict__ dZ, RowSrc src,
                                                                  float* __restrict__ part, int* err)
{
    extern __shared__ __align__(128) unsigned char tc_smem[];
    // stage b: X [16 input groups][8 row groups][8 rows][16 B], then dZ [8 output groups][8 row groups][8][16 B]
    unsigned char* Os = tc_smem + 2 * TC_WSTAGE;             // ones, the layout of X
    __shared__ __align__(8) uint64_t bar_w, bar_mma;
    __shared__ uint32_t tmem_sh;
    const int tid = threadIdx.x, warp = tid >> 5;
    bool failed = !tc_setup(&tmem_sh, &bar_w, &bar_mma, 128, nullptr, nullptr, 0);
    const uint32_t tmem = tmem_sh;
    for (int i = tid; i < TC_WCH * KIN / 8; i += TC_THREADS)   // 16 bytes of bf16 1.0 each
        *reinterpret_cast<uint4*>(Os + i * 16) = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    // M = 128 inputs, N = 64 outputs, both operands MN-major (bits 15, 16)
    constexpr uint32_t IDESC = tc_idesc_bf16(KIN, HD) | (1u << 15) | (1u << 16);
    const int nchunks = (rows + TC_WCH - 1) / TC_WCH;
    __shared__ const unsigned char* rowp[2][2][TC_WCH];       // per stage: the chunk's gathered row halves
    auto stage = [&](int c, int b) {
        unsigned char* Xs = tc_smem + b * TC_WSTAGE;
        unsigned char* Zs = Xs + TC_WCH * KIN * 2;
        const int r0 = c * TC_WCH;
        {                                                       // one index lookup per row half
            const int row = tid & (TC_WCH - 1), hf = (tid >> 6) & 1, r = r0 + row;
            if (tid < 2 * TC_WCH)
                rowp[b][hf][row] = r < rows ? reinterpret_cast<const unsigned char*>(src.half(r, hf)) : nullptr;
        }
        __syncthreads();
        for (int i = tid; i < TC_WCH * KIN / 8; i += TC_THREADS) {   // X: chunk i -> row group (i>>3)&7, inputs (i>>6)*8..
            const int row = (((i >> 3) & 7) << 3) + (i & 7), mg = i >> 6;
            const unsigned char* p = rowp[b][mg >> 3][row];
            cp_async16(Xs + i * 16, p ? p + (mg & 7) * 16 : reinterpret_cast<const unsigned char*>(dZ), p != nullptr);
        }
        for (int i = tid; i < TC_WCH * HD / 8; i += TC_THREADS) {    // dZ: outputs (i>>6)*8..
            const int r = r0 + (((i >> 3) & 7) << 3) + (i & 7), ng = i >> 6;
            const bool v = r < rows;
            const unsigned char* g = v ? reinterpret_cast<const unsigned char*>(dZ + (size_t)r * HD) + ng * 16
                                       : reinterpret_cast<const unsigned char*>(dZ);
            cp_async16(Zs + i * 16, g, v);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    uint32_t phase = 0;
    bool first = true;
    int it = 0;
    if (!failed && (int)blockIdx.x < nchunks) stage(blockIdx.x, 0);
    for (int c = blockIdx.x; !failed && c < nchunks; c += gridDim.x, ++it) {
        const int b = it & 1;
        if (c + (int)gridDim.x < nchunks) {
            stage(c + gridDim.x, b ^ 1);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
            const uint32_t xs = smem_u32(tc_smem + b * TC_WSTAGE), zs = xs + TC_WCH * KIN * 2;
#pragma unroll
            for (int ks = 0; ks < TC_WCH / 16; ++ks) {
                const uint32_t acc = (first && ks == 0) ? 0u : 1u;
                const uint64_t bz = tc_desc(zs + ks * 256, 128, 8 * 128);
                tc_mma(tmem, tc_desc(xs + ks * 256, 128, 8 * 128), bz, IDESC, acc);
                tc_mma(tmem + HD, tc_desc(smem_u32(Os) + ks * 256, 128, 8 * 128), bz, IDESC, acc);
            }
            tc_commit(&bar_mma);
        }
        first = false;
        const bool ok = mbar_wait(&bar_mma, phase);            // the chunk's MMAs are done: its stage is reusable
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (!failed) {
        tc_fence_after();
        float* P = part + (size_t)blockIdx.x * WPART;
        const int q = warp & 3, in = q * 32 + (tid & 31);      // TMEM lane = input index
        const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16);
        if (warp < 4) {
#pragma unroll
            for (int c0 = 0; c0 < HD; c0 += 16) {
                float d[16];
                tmem_ld16(tl + c0, d);
                tmem_ld_wait();
#pragma unroll
                for (int i = 0; i < 16; ++i) P[(c0 + i) * KIN + in] = d[i];
            }
        } else {
#pragma unroll
            for (int c0 = 0; c0 < HD; c0 += 16) {               // every lane holds the column sums
                float d[16];
                tmem_ld16(tl + HD + c0, d);
                tmem_ld_wait();
                if (in == 0)
#pragma unroll
                    for (int i = 0; i < 16; ++i) P[HD * KIN + c0 + i] = d[i];
            }
        }
    }
    tc_teardown(tmem, 128, failed, err);
}

// Packs the BF16 matrix W [64 outputs][128 inputs] of every layer map into the
// tcgen05 operand layouts: Wpk [8 output groups][16 k-chunks][8][8] (forward,
// B = W, K = inputs) and WTpk [16 input groups][8 k-chunks][8][8] (input
// gradient, B = W^T, K = outputs).  One thread per packed element.
__global__ void pack_weights_kernel(int nmat, const bf16* const* __restrict__ Ws, bf16* __restrict__ out)
{
    const int per = HD * KIN;
    const int64_t total = (int64_t)nmat * 2 * per;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int m = (int)(i / (2 * per)), which = (int)((i / per) & 1), e = (int)(i % per);
        const bf16* W = Ws[m];
        const int j = e & 7, r8 = (e >> 3) & 7;
        bf16 v;
        if (which == 0) {                    // output n = (e >> 10) * 8 + r8, input k = ((e >> 6) & 15) * 8 + j
            const int n = ((e >> 10) << 3) | r8, k = (((e >> 6) & 15) << 3) | j;
            v = W[n * KIN + k];
        } else {                             // input n = (e >> 9) * 8 + r8, output k = ((e >> 6) & 7) * 8 + j
            const int n = ((e >> 9) << 3) | r8, k = (((e >> 6) & 7) << 3) | j;
            v = W[k * KIN + n];
        }
        out[i] = v;
    }
}

// ------------------------------------------------------- elementwise kernels
// h0[b][n] = X[u_n]; e0[b][e] = Jt[idx(J)]
__global__ void embed_kernel(int B, int N, int E, const int* __restrict__ u, const int8_t* __restrict__ J,
                             const float* __restrict__ Xemb, const float* __restrict__ Jemb, bf16* h, bf16* e)
{
    const size_t total = (size_t)B * (N + E) * HD;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t row = i / HD;
        const int c = (int)(i % HD);
        if (row < (size_t)B * N) {
            const int n = (int)(row % N);
            h[i] = __float2bfloat16_rn(Xemb[u[n] * HD + c]);
        } else {
            const size_t re = row - (size_t)B * N;
            const int j = J[re];
            const int idx = j < 0 ? j + 3 : j + 2;          // -3,-2,-1,1,2,3 -> 0..5
            e[re * HD + c] = __float2bfloat16_rn(Jemb[idx * HD + c]);
        }
    }
}

// m[b][n] = sum over the message rows into n of R (FP32 sum, BF16 result)
__global__ void aggregate_kernel(int B, int N, int E, const int* __restrict__ in_rows, const float* __restrict__ R, bf16* m)
{
    const size_t total = (size_t)B * N * (HD / 2);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t bn = i / (HD / 2);
        const int cp = (int)(i % (HD / 2));
        const int b = (int)(bn / N), n = (int)(bn % N);
        float x = 0.f, y = 0.f;
        for (int s = 0; s < MAXDEG; ++s) {
            const int r = in_rows[n * MAXDEG + s];
            if (r < 0) continue;
            const float2 v = reinterpret_cast<const float2*>(R + ((size_t)b * 2 * E + r) * HD)[cp];
            x += v.x;
            y += v.y;
        }
        reinterpret_cast<uint32_t*>(m + bn * HD)[cp] = pack_bf2(x, y);
    }
}

// s[b][e] = h[b][ei] + h[b][ej]
__global__ void endpoint_sum_kernel(int B, int N, int E, const int* __restrict__ ei, const int* __restrict__ ej,
                                    const bf16* __restrict__ h, bf16* s)
{
    const size_t total = (size_t)B * E * (HD / 2);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t be = i / (HD / 2);
        const int cp = (int)(i % (HD / 2));
        const int b = (int)(be / E), e = (int)(be % E);
        const float2 x = unpack_bf2(reinterpret_cast<const uint32_t*>(h + ((size_t)b * N + ei[e]) * HD)[cp]);
        const float2 y = unpack_bf2(reinterpret_cast<const uint32_t*>(h + ((size_t)b * N + ej[e]) * HD)[cp]);
        reinterpret_cast<uint32_t*>(s + be * HD)[cp] = pack_bf2(x.x + y.x, x.y + y.y);
    }
}

// dZ[r] = G[gidx(r)] * (Z[r] > 0) as BF16.  gmap (optional) sends row r to
// gradient row (r / R_local) * S + gmap[r % R_local].
__global__ void relu_mask_kernel(int rows, const float* __restrict__ G, const int* __restrict__ gmap, int R_local, int S,
                                 const bf16* __restrict__ Z, bf16* dZ)
{
    const size_t total = (size_t)rows * (HD / 2);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / (HD / 2)), cp = (int)(i % (HD / 2));
        size_t gr = r;
        if (gmap) gr = (size_t)(r / R_local) * S + gmap[r % R_local];
        const float2 gv = reinterpret_cast<const float2*>(G + gr * HD)[cp];
        const float2 z = unpack_bf2(reinterpret_cast<const uint32_t*>(Z + (size_t)r * HD)[cp]);
        reinterpret_cast<uint32_t*>(dZ + (size_t)r * HD)[cp] = pack_bf2(z.x > 0.f ? gv.x : 0.f, z.y > 0.f ? gv.y : 0.f);
    }
}

// out[b][n] += sum over list[n][0..5] (>= 0) of src[b][list][off..off+63] (src rows of width `w`)
__global__ void gather_add_kernel(int B, int N, int Rsrc, const int* __restrict__ list, const float* __restrict__ src,
                                  int w, int off, float* out)
{
    const size_t total = (size_t)B * N * HD;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t bn = i / HD;
        const int c = (int)(i % HD);
        const int b = (int)(bn / N), n = (int)(bn % N);
        float acc = 0.f;
        for (int s = 0; s < MAXDEG; ++s) {
            const int r = list[n * MAXDEG + s];
            if (r >= 0) acc += src[((size_t)b * Rsrc + r) * w + off + c];
        }
        out[i] += acc;
    }
}

// readout forward + loss gradient (one block per graph, HD threads)
__global__ void readout_kernel(int N, const bf16* __restrict__ h, const float* __restrict__ W1, const float* __restrict__ b1,
                               const float* __restrict__ w2, const float* __restrict__ b2, float* y, float* gbuf,
                               float* zbuf, const float* __restrict__ target, float inv_B, float* dybuf,
                               float* sqbuf, float* dh)
{
    __shared__ float gs[HD], as[HD], red[HD], dz[HD];
    const int b = blockIdx.x, c = threadIdx.x;
    float acc = 0.f;
    for (int n = 0; n < N; ++n) acc += __bfloat162float(h[((size_t)b * N + n) * HD + c]);
    gs[c] = acc / (float)N;
    __syncthreads();
    float z = b1[c];
    for (int k = 0; k < HD; ++k) z += W1[c * HD + k] * gs[k];
    as[c] = fmaxf(z, 0.f);
    red[c] = as[c] * w2[c];
    gbuf[b * HD + c] = gs[c];
    zbuf[b * HD + c] = z;
    __syncthreads();
    for (int s = HD / 2; s > 0; s >>= 1) {
        if (c < s) red[c] += red[c + s];
        __syncthreads();
    }
    const float yb = red[0] + b2[0];
    if (c == 0) y[b] = yb;
    if (!target) return;
    const float dy = 2.f * (yb - target[b]) * inv_B;
    if (c == 0) {                                  // this graph's loss term and output gradient (summed in order
        dybuf[b] = dy;                             // over graphs by readout_grad_kernel)
        sqbuf[b] = (yb - target[b]) * (yb - target[b]) * inv_B;
    }
    dz[c] = z > 0.f ? dy * w2[c] : 0.f;
    __syncthreads();
    float dg = 0.f;
    for (int o = 0; o < HD; ++o) dg += dz[o] * W1[o * HD + c];
    dg /= (float)N;
    for (int n = 0; n < N; ++n) dh[((size_t)b * N + n) * HD + c] = dg;
}

// Readout parameter gradients and the loss, summed over the B graphs in graph
// order (bit-reproducible): block c < 64, thread k: dW1[c][k] += sum_b dz_b[c]
// g_b[k] with dz_b[c] = dy_b w2[c] where z_b[c] > 0, and (thread 0) db1[c],
// dw2[c]; block 64: db2 and the loss.
__global__ void readout_grad_kernel(int B, const float* __restrict__ gbuf, const float* __restrict__ zbuf,
                                    const float* __restrict__ dybuf, const float* __restrict__ sqbuf,
                                    const float* __restrict__ w2, float* loss, float* dW1, float* db1, float* dw2,
                                    float* db2)
{
    const int c = blockIdx.x, k = threadIdx.x;
    if (c < HD) {
        const float w = w2[c];
        float acc = 0.f, a1 = 0.f, a2 = 0.f;
        for (int b = 0; b < B; ++b) {
            const float z = zbuf[b * HD + c], dy = dybuf[b];
            const float dz = z > 0.f ? dy * w : 0.f;
            acc += dz * gbuf[b * HD + k];
            a1 += dz;
            a2 += dy * fmaxf(z, 0.f);
        }
        dW1[c * HD + k] += acc;
        if (k == 0) {
            db1[c] += a1;
            dw2[c] += a2;
        }
    } else if (k == 0) {
        float s2 = 0.f, l = 0.f;
        for (int b = 0; b < B; ++b) {
            s2 += dybuf[b];
            l += sqbuf[b];
        }
        db2[0] += s2;
        *loss += l;
    }
}

// Embedding gradients: dX[o] += sum of dh over the nodes of orientation o, dJt[v] += sum of de over
// the edges of coupler value v.  A thread owns column c of a strided set of rows and keeps its 2 + 6
// class sums in registers; the block adds its 4 lanes' sums in lane order and writes them as its
// partial part[block][8][64] (classes: orientations 0, 1, coupler values -3..3 without 0), and
// embed_bwd_reduce adds the partials in block order (bit-reproducible).  256 threads per block.
__global__ void embed_bwd_kernel(int B, int N, int E, const int* __restrict__ u, const int8_t* __restrict__ J,
                                 const float* __restrict__ dh, const float* __restrict__ de, float* __restrict__ part)
{
    __shared__ float sp[4][8][HD];
    const int c = threadIdx.x % HD, lane = threadIdx.x / HD, lanes = blockDim.x / HD;
    const size_t nN = (size_t)B * N, nE = (size_t)B * E, stride = (size_t)gridDim.x * lanes;
    const size_t first = blockIdx.x * (size_t)lanes + lane;
    float ax0 = 0.f, ax1 = 0.f, aj[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (size_t row = first; row < nN; row += stride) {
        const float v = dh[row * HD + c];
        if (u[row % N]) ax1 += v;
        else ax0 += v;
    }
    for (size_t re = first; re < nE; re += stride) {
        const int j = J[re];
        const int k = j < 0 ? j + 3 : j + 2;                 // -3,-2,-1,1,2,3 -> 0..5
        const float v = de[re * HD + c];
#pragma unroll
        for (int q = 0; q < 6; ++q) aj[q] += k == q ? v : 0.f;
    }
    sp[lane][0][c] = ax0;
    sp[lane][1][c] = ax1;
#pragma unroll
    for (int q = 0; q < 6; ++q) sp[lane][2 + q][c] = aj[q];
    __syncthreads();
    for (int i = threadIdx.x; i < 8 * HD; i += blockDim.x) {
        float t = 0.f;
        for (int l = 0; l < lanes; ++l) t += sp[l][i / HD][i % HD];
        part[(size_t)blockIdx.x * 8 * HD + i] = t;
    }
}

__global__ void embed_bwd_reduce(int nblocks, const float* __restrict__ part, float* dX, float* dJt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 8 * HD) return;
    float t = 0.f;
    for (int b = 0; b < nblocks; ++b) t += part[(size_t)b * 8 * HD + i];
    if (i < 2 * HD) dX[i] += t;
    else dJt[i - 2 * HD] += t;
}

__global__ void adam_kernel(int64_t n, float* theta, const float* __restrict__ g, float* m, float* v, float lr,
                            float b1, float b2, float c1, float c2, float eps)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

__global__ void to_bf16_kernel(int64_t n, const float* __restrict__ x, bf16* y)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16_rn(x[i]);
}

int grid_for(size_t work, int block = 256)
{
    const size_t b = (work + block - 1) / block;
    return (int)(b > 8192 ? 8192 : (b < 1 ? 1 : b));
}

}  // namespace

// ==========================================================================
// host runtime
// ==========================================================================
struct sg_model {
    int layers = 4;
    int64_t nparams = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    float *theta = nullptr, *grad = nullptr, *mom1 = nullptr, *mom2 = nullptr, *dloss = nullptr;
    bf16* wbf = nullptr;          // BF16 copy of theta
    bf16* wpk = nullptr;          // per layer map: W and W^T in the tcgen05 operand layouts (2 x 8192 BF16 each)
    const bf16** d_wptr = nullptr;// device array: the BF16 matrices of every layer map (pack_weights_kernel input)
    int* d_err = nullptr;         // set by a tensor-core kernel whose bounded wait ran out
    int sms = 0;                  // SMs of the device (persistent grids)
    int64_t step = 0;
    // offsets into theta
    int64_t oX = 0, oJ = 0, oW1 = 0, ob1 = 0, ow2 = 0, ob2 = 0;
    std::vector<int64_t> oWm, obm, oWu, obu, oWe, obe;
    // graph + activation buffers for the current (L, Bcap)
    int L = 0, N = 0, E = 0, Bcap = 0;
    int *d_u = nullptr, *d_ei = nullptr, *d_ej = nullptr, *d_in_rows = nullptr, *d_out_rows = nullptr,
        *d_inc = nullptr, *d_src = nullptr, *d_tgt = nullptr, *d_eid = nullptr, *d_iden = nullptr, *d_msg_edge = nullptr;
    int8_t* d_J = nullptr;
    float *d_t = nullptr, *d_y = nullptr, *d_g = nullptr, *d_z = nullptr;
    float *d_dy = nullptr, *d_sq = nullptr;   // per graph: output gradient, loss term (readout)
    float* d_epart = nullptr;                 // embedding-gradient block partials [4 x SMs][8][64]
    std::vector<bf16*> h, e, m, s, zm, zu, ze;
    float *R = nullptr, *dX = nullptr, *dh = nullptr, *dh2 = nullptr, *de = nullptr, *dm = nullptr, *ds = nullptr;
    bf16* dZ = nullptr;
    float* wpart = nullptr;       // weight-gradient partials, one WPART block per persistent CTA
    float* wred = nullptr;        // [WRED_GROUPS][WPART] group sums of the partials
    int wblocks = 0;              // persistent CTAs of the weight-gradient kernel
    uint64_t launches = 0;
    std::string err = "no error";
};

namespace {

int sfail(sg_model* m, int code, const std::string& msg)
{
    if (m) m->err = msg;
    else ptg::set_global_error(msg.c_str());
    return code;
}

#define SK(call, what)                                                                              \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            return sfail(M, e_ == cudaErrorMemoryAllocation ? PT_ERR_OOM : PT_ERR_CUDA,             \
                         std::string(what) + ": " + cudaGetErrorString(e_));                        \
    } while (0)

template <class T>
cudaError_t salloc(T** p, size_t n)
{
    return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (n ? n : 1));
}

void free_graph(sg_model* M)
{
    int** ints[] = {&M->d_u, &M->d_ei, &M->d_ej, &M->d_in_rows, &M->d_out_rows, &M->d_inc, &M->d_src, &M->d_tgt,
                    &M->d_eid, &M->d_iden, &M->d_msg_edge};
    for (int** p : ints) { cudaFree(*p); *p = nullptr; }
    cudaFree(M->d_J); M->d_J = nullptr;
    float** fl[] = {&M->d_t, &M->d_y, &M->d_g, &M->d_z, &M->d_dy, &M->d_sq, &M->d_epart, &M->R, &M->dX, &M->dh,
                    &M->dh2, &M->de, &M->dm, &M->ds};
    for (float** p : fl) { cudaFree(*p); *p = nullptr; }
    cudaFree(M->dZ); M->dZ = nullptr;
    cudaFree(M->wpart); M->wpart = nullptr;
    cudaFree(M->wred); M->wred = nullptr;
    for (auto* v : {&M->h, &M->e, &M->m, &M->s, &M->zm, &M->zu, &M->ze}) {
        for (bf16* p : *v) cudaFree(p);
        v->clear();
    }
    M->L = M->Bcap = 0;
}

// Builds the Chimera C_L topology in the coupler order of pt.h and sizes the
// activation buffers for B graphs.
int prepare(sg_model* M, int L, int B)
{
    if (M->L == L && M->Bcap >= B) return PT_OK;
    free_graph(M);
    const int N = 8 * L * L, E = 16 * L * L + 8 * L * (L - 1);
    std::vector<int> ei, ej;
    auto idx = [L](int r, int c, int u, int k) { return 8 * (r * L + c) + 4 * u + k; };
    for (int r = 0; r < L; ++r)
        for (int c = 0; c < L; ++c)
            for (int k = 0; k < 4; ++k)
                for (int kp = 0; kp < 4; ++kp) { ei.push_back(idx(r, c, 0, k)); ej.push_back(idx(r, c, 1, kp)); }
    for (int r = 0; r + 1 < L; ++r)
        for (int c = 0; c < L; ++c)
            for (int k = 0; k < 4; ++k) { ei.push_back(idx(r, c, 0, k)); ej.push_back(idx(r + 1, c, 0, k)); }
    for (int r = 0; r < L; ++r)
        for (int c = 0; c + 1 < L; ++c)
            for (int k = 0; k < 4; ++k) { ei.push_back(idx(r, c, 1, k)); ej.push_back(idx(r, c + 1, 1, k)); }
    // message row 2e: source ej -> target ei; row 2e+1: source ei -> target ej
    std::vector<int> u(N), src(2 * E), tgt(2 * E), eid(2 * E), iden(std::max(N, 2 * E));
    std::vector<int> in_rows(N * MAXDEG, -1), out_rows(N * MAXDEG, -1), inc(N * MAXDEG, -1);
    std::vector<int> cin(N, 0), cout(N, 0), cinc(N, 0);
    for (int i = 0; i < N; ++i) u[i] = (i >> 2) & 1;
    for (int q = 0; q < (int)iden.size(); ++q) iden[q] = q;
    for (int e2 = 0; e2 < E; ++e2) {
        src[2 * e2] = ej[e2]; tgt[2 * e2] = ei[e2];
        src[2 * e2 + 1] = ei[e2]; tgt[2 * e2 + 1] = ej[e2];
        eid[2 * e2] = eid[2 * e2 + 1] = e2;
        for (int d = 0; d < 2; ++d) {
            const int r = 2 * e2 + d;
            in_rows[tgt[r] * MAXDEG + cin[tgt[r]]++] = r;
            out_rows[src[r] * MAXDEG + cout[src[r]]++] = r;
        }
        inc[ei[e2] * MAXDEG + cinc[ei[e2]]++] = e2;
        inc[ej[e2] * MAXDEG + cinc[ej[e2]]++] = e2;
    }
    auto up = [&](int** d, const std::vector<int>& v) -> cudaError_t {
        cudaError_t r = salloc(d, v.size());
        if (r != cudaSuccess) return r;
        return cudaMemcpy(*d, v.data(), 4 * v.size(), cudaMemcpyHostToDevice);
    };
    SK(up(&M->d_u, u), "upload topology");
    SK(up(&M->d_ei, ei), "upload topology");
    SK(up(&M->d_ej, ej), "upload topology");
    SK(up(&M->d_in_rows, in_rows), "upload topology");
    SK(up(&M->d_out_rows, out_rows), "upload topology");
    SK(up(&M->d_inc, inc), "upload topology");
    SK(up(&M->d_src, src), "upload topology");
    SK(up(&M->d_tgt, tgt), "upload topology");
    SK(up(&M->d_eid, eid), "upload topology");
    SK(up(&M->d_iden, iden), "upload topology");
    const size_t nN = (size_t)B * N, nE = (size_t)B * E, nM = 2 * nE;
    SK(salloc(&M->d_J, nE), "cudaMalloc J");
    SK(salloc(&M->d_t, (size_t)B), "cudaMalloc t");
    SK(salloc(&M->d_y, (size_t)B), "cudaMalloc y");
    SK(salloc(&M->d_g, (size_t)B * HD), "cudaMalloc g");
    SK(salloc(&M->d_z, (size_t)B * HD), "cudaMalloc z");
    SK(salloc(&M->d_dy, (size_t)B), "cudaMalloc dy");
    SK(salloc(&M->d_sq, (size_t)B), "cudaMalloc sq");
    SK(salloc(&M->d_epart, (size_t)4 * M->sms * 8 * HD), "cudaMalloc embedding partials");
    M->h.assign(M->layers + 1, nullptr);
    M->e.assign(M->layers + 1, nullptr);
    M->m.assign(M->layers, nullptr);
    M->s.assign(M->layers, nullptr);
    M->zm.assign(M->layers, nullptr);
    M->zu.assign(M->layers, nullptr);
    M->ze.assign(M->layers, nullptr);
    for (int l = 0; l <= M->layers; ++l) {
        SK(salloc(&M->h[l], nN * HD), "cudaMalloc h");
        SK(salloc(&M->e[l], nE * HD), "cudaMalloc e");
    }
    for (int l = 0; l < M->layers; ++l) {
        SK(salloc(&M->m[l], nN * HD), "cudaMalloc m");
        SK(salloc(&M->s[l], nE * HD), "cudaMalloc s");
        SK(salloc(&M->zm[l], nM * HD), "cudaMalloc zm");
        SK(salloc(&M->zu[l], nN * HD), "cudaMalloc zu");
        SK(salloc(&M->ze[l], nE * HD), "cudaMalloc ze");
    }
    SK(salloc(&M->R, nM * HD), "cudaMalloc R");
    SK(salloc(&M->dX, nM * HD), "cudaMalloc dX");           // message rows' node half of the input gradient
    SK(salloc(&M->dZ, nM * HD), "cudaMalloc dZ");
    {
        int dev = 0, sms = 0;
        SK(cudaGetDevice(&dev), "cudaGetDevice");
        SK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device attribute");
        M->wblocks = TC_CTAS_WGRAD * sms;     // persistent weight-gradient CTAs
        SK(salloc(&M->wpart, (size_t)M->wblocks * WPART), "cudaMalloc wpart");
        SK(salloc(&M->wred, (size_t)WRED_GROUPS * WPART), "cudaMalloc wred");
    }
    SK(salloc(&M->dh, nN * HD), "cudaMalloc dh");
    SK(salloc(&M->dh2, nN * HD), "cudaMalloc dh2");
    SK(salloc(&M->dm, nN * HD), "cudaMalloc dm");
    SK(salloc(&M->de, nE * HD), "cudaMalloc de");
    SK(salloc(&M->ds, nE * HD), "cudaMalloc ds");
    M->L = L; M->N = N; M->E = E; M->Bcap = B;
    return PT_OK;
}

RowSrc rows_of(const bf16* P0, const int* map0, int S0, const bf16* P1, const int* map1, int S1, int R_local)
{
    RowSrc r;
    r.P0 = P0; r.map0 = map0; r.S0 = S0; r.P1 = P1; r.map1 = map1; r.S1 = S1; r.R_local = R_local;
    return r;
}

// The tcgen05 operand copies of every layer matrix follow the BF16 weights.
void pack_weights(sg_model* M)
{
    pack_weights_kernel<<<grid_for((size_t)M->layers * 3 * 2 * HD * KIN), 256, 0, M->stream>>>(M->layers * 3,
                                                                                                  M->d_wptr, M->wpk);
    M->launches++;
}

// Packed operands of layer l's map `which` (0 messages, 1 node update, 2 edge update).
const bf16* wpk_fwd(const sg_model* M, int l, int which) { return M->wpk + ((size_t)(l * 3 + which) * 2) * HD * KIN; }
const bf16* wpk_bwd(const sg_model* M, int l, int which) { return wpk_fwd(M, l, which) + HD * KIN; }

int tc_grid(const sg_model* M, int rows, int ctas_per_sm)
{
    const int tiles = (rows + TC_ROWS - 1) / TC_ROWS, cap = ctas_per_sm * M->sms;
    return tiles < cap ? (tiles > 0 ? tiles : 1) : cap;
}


// dW += dZ^T X, db += column sums of dZ over `rows` rows (two launches).
void lin_wgrad(sg_model* M, int rows, const RowSrc& src, float* dW, float* db)
{
    const int nchunks = (rows + TC_WCH - 1) / TC_WCH;
    const int grid = nchunks < M->wblocks ? (nchunks > 0 ? nchunks : 1) : M->wblocks;
    lin_wgrad_tc_kernel<<<grid, TC_THREADS, TC_SMEM_WGRAD, M->stream>>>(rows, M->dZ, src, M->wpart, M->d_err);
    lin_wgrad_reduce1<<<dim3((WPART + 255) / 256, WRED_GROUPS), 256, 0, M->stream>>>(grid, M->wpart, M->wred);
    lin_wgrad_reduce2<<<(WPART + 255) / 256, 256, 0, M->stream>>>(M->wred, dW, db);
}

int forward(sg_model* M, int B, bool train)
{
    const int N = M->N, E = M->E;
    cudaStream_t st = M->stream;
    embed_kernel<<<grid_for((size_t)B * (N + E) * HD), 256, 0, st>>>(B, N, E, M->d_u, M->d_J, M->theta + M->oX,
                                                                       M->theta + M->oJ, M->h[0], M->e[0]);
    M->launches++;
    for (int l = 0; l < M->layers; ++l) {
        // messages: row 2e / 2e+1 of every graph: [h[src] | e[edge]]
        const RowSrc ms = rows_of(M->h[l], M->d_src, N, M->e[l], M->d_eid, E, 2 * E);
        lin_fwd_tc_kernel<0><<<tc_grid(M, B * 2 * E, TC_CTAS_FWD), TC_THREADS, TC_SMEM_FWD, st>>>(B * 2 * E, ms, wpk_fwd(M, l, 0),
                                                                           M->theta + M->obm[l], M->zm[l], M->R,
                                                                           nullptr, M->d_err);
        aggregate_kernel<<<grid_for((size_t)B * N * HD / 2), 256, 0, st>>>(B, N, E, M->d_in_rows, M->R, M->m[l]);
        const RowSrc ns = rows_of(M->h[l], M->d_iden, N, M->m[l], M->d_iden, N, N);
        lin_fwd_tc_kernel<1><<<tc_grid(M, B * N, TC_CTAS_FWD), TC_THREADS, TC_SMEM_FWD, st>>>(B * N, ns, wpk_fwd(M, l, 1), M->theta + M->obu[l],
                                                                       M->zu[l], nullptr, M->h[l + 1], M->d_err);
        endpoint_sum_kernel<<<grid_for((size_t)B * E * HD / 2), 256, 0, st>>>(B, N, E, M->d_ei, M->d_ej, M->h[l + 1], M->s[l]);
        const RowSrc es = rows_of(M->e[l], M->d_iden, E, M->s[l], M->d_iden, E, E);
        lin_fwd_tc_kernel<1><<<tc_grid(M, B * E, TC_CTAS_FWD), TC_THREADS, TC_SMEM_FWD, st>>>(B * E, es, wpk_fwd(M, l, 2), M->theta + M->obe[l],
                                                                       M->ze[l], nullptr, M->e[l + 1], M->d_err);
        M->launches += 5;
    }
    (void)train;
    return PT_OK;
}

// Gradient of the mean squared error into M->grad (zeroed first); loss into M->dloss.
int backward_all(sg_model* M, int B)
{
    const int N = M->N, E = M->E;
    cudaStream_t st = M->stream;
    float* G = M->grad;
    SK(cudaMemsetAsync(G, 0, sizeof(float) * M->nparams, st), "zero grad");
    SK(cudaMemsetAsync(M->dloss, 0, sizeof(float), st), "zero loss");
    SK(cudaMemsetAsync(M->de, 0, sizeof(float) * (size_t)B * E * HD, st), "zero de");
    readout_kernel<<<B, HD, 0, st>>>(N, M->h[M->layers], M->theta + M->oW1, M->theta + M->ob1, M->theta + M->ow2,
                                     M->theta + M->ob2, M->d_y, M->d_g, M->d_z, M->d_t, 1.f / (float)B, M->d_dy,
                                     M->d_sq, M->dh);
    readout_grad_kernel<<<HD + 1, HD, 0, st>>>(B, M->d_g, M->d_z, M->d_dy, M->d_sq, M->theta + M->ow2, M->dloss,
                                               G + M->oW1, G + M->ob1, G + M->ow2, G + M->ob2);
    M->launches += 2;
    const size_t nN = (size_t)B * N, nE = (size_t)B * E;
    for (int l = M->layers - 1; l >= 0; --l) {
        // edge update: e' = e + relu(ze), ze = We [e | s] + be
        relu_mask_kernel<<<grid_for(nE * HD / 2), 256, 0, st>>>(B * E, M->de, nullptr, 1, 1, M->ze[l], M->dZ);
        // de += dX[:, :64] (into e), ds = dX[:, 64:]
        lin_bwd_input_tc_kernel<1><<<tc_grid(M, B * E, TC_CTAS_BWD), TC_THREADS, TC_SMEM_BWD, st>>>(B * E, M->dZ, wpk_bwd(M, l, 2), nullptr,
                                                                             M->de, M->de, M->ds, M->d_err);
        const RowSrc es = rows_of(M->e[l], M->d_iden, E, M->s[l], M->d_iden, E, E);
        lin_wgrad(M, B * E, es, G + M->oWe[l], G + M->obe[l]);
        SK(cudaMemcpyAsync(M->dh2, M->dh, sizeof(float) * nN * HD, cudaMemcpyDeviceToDevice, st), "copy dh");
        gather_add_kernel<<<grid_for(nN * HD), 256, 0, st>>>(B, N, E, M->d_inc, M->ds, HD, 0, M->dh2);
        // node update: h' = h + relu(zu), zu = Wu [h | m] + bu
        relu_mask_kernel<<<grid_for(nN * HD / 2), 256, 0, st>>>(B * N, M->dh2, nullptr, 1, 1, M->zu[l], M->dZ);
        // dh = dh2 + dX[:, :64] (into h), dm = dX[:, 64:]
        lin_bwd_input_tc_kernel<1><<<tc_grid(M, B * N, TC_CTAS_BWD), TC_THREADS, TC_SMEM_BWD, st>>>(B * N, M->dZ, wpk_bwd(M, l, 1), nullptr,
                                                                             M->dh2, M->dh, M->dm, M->d_err);
        const RowSrc ns = rows_of(M->h[l], M->d_iden, N, M->m[l], M->d_iden, N, N);
        lin_wgrad(M, B * N, ns, G + M->oWu[l], G + M->obu[l]);
        // messages: m_i = sum relu(zm) over rows into i
        relu_mask_kernel<<<grid_for(nE * 2 * HD / 2), 256, 0, st>>>(B * 2 * E, M->dm, M->d_tgt, 2 * E, N, M->zm[l], M->dZ);
        lin_bwd_input_tc_kernel<0><<<tc_grid(M, B * 2 * E, TC_CTAS_BWD), TC_THREADS, TC_SMEM_BWD, st>>>(B * 2 * E, M->dZ, wpk_bwd(M, l, 0),
                                                                                 M->dX, nullptr, nullptr, M->de,
                                                                                 M->d_err);
        const RowSrc ms = rows_of(M->h[l], M->d_src, N, M->e[l], M->d_eid, E, 2 * E);
        lin_wgrad(M, B * 2 * E, ms, G + M->oWm[l], G + M->obm[l]);
        gather_add_kernel<<<grid_for(nN * HD), 256, 0, st>>>(B, N, 2 * E, M->d_out_rows, M->dX, HD, 0, M->dh);
        M->launches += 17;
    }
    embed_bwd_kernel<<<4 * M->sms, 256, 0, st>>>(B, N, E, M->d_u, M->d_J, M->dh, M->de, M->d_epart);
    embed_bwd_reduce<<<(8 * HD + 255) / 256, 256, 0, st>>>(4 * M->sms, M->d_epart, G + M->oX, G + M->oJ);
    M->launches += 2;
    return PT_OK;
}

// A tensor-core kernel whose bounded mbarrier wait ran out leaves 1 in d_err
// (its CTA stopped and freed its tensor memory): the call reports a timeout
// and the word is cleared for the next call.
int tc_status(sg_model* M, int terr)
{
    if (!terr) return PT_OK;
    SK(cudaMemsetAsync(M->d_err, 0, sizeof(int), M->stream), "clear status");
    SK(cudaStreamSynchronize(M->stream), "sync status");
    return sfail(M, PT_ERR_TIMEOUT, "a tensor-core kernel's mbarrier wait ran out (results of this call are invalid)");
}

int load_batch(sg_model* M, int L, int B, const int8_t* J, const float* t)
{
    if (L < 1 || L > ptg::MAX_L || B < 1 || B > 4096 || !J) return sfail(M, PT_ERR_ARG, "need 1 <= L <= 16, 1 <= B <= 4096");
    const int E = 16 * L * L + 8 * L * (L - 1);
    for (size_t i = 0; i < (size_t)B * E; ++i)
        if (J[i] == 0 || J[i] < -3 || J[i] > 3) return sfail(M, PT_ERR_ARG, "surrogate couplers must be in {+-1, +-2, +-3}");
    int rc = prepare(M, L, B);
    if (rc) return rc;
    SK(cudaMemcpyAsync(M->d_J, J, (size_t)B * E, cudaMemcpyHostToDevice, M->stream), "upload J");
    if (t) SK(cudaMemcpyAsync(M->d_t, t, sizeof(float) * B, cudaMemcpyHostToDevice, M->stream), "upload targets");
    return PT_OK;
}

}  // namespace

extern "C" {

const char* sg_last_error(const sg_model* m) { return m ? m->err.c_str() : pt_last_error(nullptr); }

int sg_create(sg_model** out, int32_t hidden, int32_t layers, void* stream)
{
    sg_model* M = nullptr;
    if (!out) return sfail(nullptr, PT_ERR_ARG, "NULL argument");
    *out = nullptr;
    if (hidden != HD || layers < 1 || layers > 8) return sfail(nullptr, PT_ERR_ARG, "hidden must be 64, layers in [1, 8]");
    M = new (std::nothrow) sg_model();
    if (!M) return sfail(nullptr, PT_ERR_OOM, "host allocation failed");
    M->layers = layers;
    int64_t o = 0;
    M->oX = o; o += 2 * HD;
    M->oJ = o; o += 6 * HD;
    for (int l = 0; l < layers; ++l) {
        M->oWm.push_back(o); o += HD * KIN;
        M->obm.push_back(o); o += HD;
        M->oWu.push_back(o); o += HD * KIN;
        M->obu.push_back(o); o += HD;
        M->oWe.push_back(o); o += HD * KIN;
        M->obe.push_back(o); o += HD;
    }
    M->oW1 = o; o += HD * HD;
    M->ob1 = o; o += HD;
    M->ow2 = o; o += HD;
    M->ob2 = o; o += 1;
    M->nparams = o;
    auto bail = [&](int code) { std::string msg = M->err; sg_destroy(M); return sfail(nullptr, code, msg); };
    if (stream) M->stream = (cudaStream_t)stream;
    else {
        cudaError_t e = cudaStreamCreateWithFlags(&M->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { M->err = std::string("cudaStreamCreate: ") + cudaGetErrorString(e); return bail(PT_ERR_CUDA); }
        M->own_stream = true;
    }
    if (salloc(&M->theta, o) != cudaSuccess || salloc(&M->grad, o) != cudaSuccess || salloc(&M->mom1, o) != cudaSuccess ||
        salloc(&M->mom2, o) != cudaSuccess || salloc(&M->wbf, o) != cudaSuccess || salloc(&M->dloss, 1) != cudaSuccess) {
        M->err = "cudaMalloc parameters failed";
        return bail(PT_ERR_OOM);
    }
    cudaMemset(M->theta, 0, sizeof(float) * o);
    cudaMemset(M->mom1, 0, sizeof(float) * o);
    cudaMemset(M->mom2, 0, sizeof(float) * o);
    cudaMemset(M->wbf, 0, sizeof(bf16) * o);
    {
        // tcgen05 operand copies of the layer matrices, their source pointers, the timeout word
        std::vector<const bf16*> ptrs;
        for (int l = 0; l < layers; ++l) {
            ptrs.push_back(M->wbf + M->oWm[l]);
            ptrs.push_back(M->wbf + M->oWu[l]);
            ptrs.push_back(M->wbf + M->oWe[l]);
        }
        int dev = 0, sms = 0;
        if (salloc(&M->wpk, (size_t)layers * 3 * 2 * HD * KIN) != cudaSuccess ||
            salloc(&M->d_wptr, ptrs.size()) != cudaSuccess || salloc(&M->d_err, 1) != cudaSuccess) {
            M->err = "cudaMalloc tensor-core operands failed";
            return bail(PT_ERR_OOM);
        }
        cudaError_t e = cudaMemcpy(M->d_wptr, ptrs.data(), sizeof(bf16*) * ptrs.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(M->wpk, 0, sizeof(bf16) * (size_t)layers * 3 * 2 * HD * KIN);
        if (e == cudaSuccess) e = cudaMemset(M->d_err, 0, sizeof(int));
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const void* tk[5] = {(const void*)lin_fwd_tc_kernel<0>, (const void*)lin_fwd_tc_kernel<1>,
                             (const void*)lin_bwd_input_tc_kernel<0>, (const void*)lin_bwd_input_tc_kernel<1>,
                             (const void*)lin_wgrad_tc_kernel};
        const int sm_bytes[5] = {TC_SMEM_FWD, TC_SMEM_FWD, TC_SMEM_BWD, TC_SMEM_BWD, TC_SMEM_WGRAD};
        for (int q = 0; q < 5; ++q)
            if (e == cudaSuccess) e = cudaFuncSetAttribute(tk[q], cudaFuncAttributeMaxDynamicSharedMemorySize, sm_bytes[q]);
        if (e != cudaSuccess) {
            M->err = std::string("tensor-core set-up: ") + cudaGetErrorString(e);
            return bail(PT_ERR_CUDA);
        }
        M->sms = sms;
    }
    *out = M;
    return PT_OK;
}

void sg_destroy(sg_model* M)
{
    if (!M) return;
    if (M->stream) cudaStreamSynchronize(M->stream);
    free_graph(M);
    cudaFree(M->theta); cudaFree(M->grad); cudaFree(M->mom1); cudaFree(M->mom2); cudaFree(M->wbf); cudaFree(M->dloss);
    cudaFree(M->wpk); cudaFree(M->d_wptr); cudaFree(M->d_err);
    if (M->own_stream && M->stream) cudaStreamDestroy(M->stream);
    delete M;
}

int64_t sg_num_params(const sg_model* M) { return M ? M->nparams : 0; }

int sg_set_params(sg_model* M, const float* theta)
{
    if (!M || !theta) return sfail(M, PT_ERR_ARG, "NULL argument");
    SK(cudaMemcpyAsync(M->theta, theta, sizeof(float) * M->nparams, cudaMemcpyHostToDevice, M->stream), "upload params");
    SK(cudaMemsetAsync(M->mom1, 0, sizeof(float) * M->nparams, M->stream), "zero moments");
    SK(cudaMemsetAsync(M->mom2, 0, sizeof(float) * M->nparams, M->stream), "zero moments");
    to_bf16_kernel<<<grid_for((size_t)M->nparams), 256, 0, M->stream>>>(M->nparams, M->theta, M->wbf);
    M->launches++;
    pack_weights(M);
    M->step = 0;
    SK(cudaStreamSynchronize(M->stream), "sync set_params");
    return PT_OK;
}

int sg_get_params(sg_model* M, float* theta)
{
    if (!M || !theta) return sfail(M, PT_ERR_ARG, "NULL argument");
    SK(cudaMemcpyAsync(theta, M->theta, sizeof(float) * M->nparams, cudaMemcpyDeviceToHost, M->stream), "download params");
    SK(cudaStreamSynchronize(M->stream), "sync get_params");
    return PT_OK;
}

int sg_forward(sg_model* M, int32_t L, int32_t B, const int8_t* J, float* y)
{
    if (!M || !y) return sfail(M, PT_ERR_ARG, "NULL argument");
    int rc = load_batch(M, L, B, J, nullptr);
    if (rc) return rc;
    if ((rc = forward(M, B, false))) return rc;
    readout_kernel<<<B, HD, 0, M->stream>>>(M->N, M->h[M->layers], M->theta + M->oW1, M->theta + M->ob1,
                                            M->theta + M->ow2, M->theta + M->ob2, M->d_y, M->d_g, M->d_z, nullptr,
                                            0.f, nullptr, nullptr, nullptr);
    M->launches++;
    SK(cudaGetLastError(), "forward kernels");
    SK(cudaMemcpyAsync(y, M->d_y, sizeof(float) * B, cudaMemcpyDeviceToHost, M->stream), "download y");
    int terr = 0;
    SK(cudaMemcpyAsync(&terr, M->d_err, sizeof(int), cudaMemcpyDeviceToHost, M->stream), "download status");
    SK(cudaStreamSynchronize(M->stream), "sync forward");
    return tc_status(M, terr);
}

int sg_grad(sg_model* M, int32_t L, int32_t B, const int8_t* J, const float* t, float* loss, float* grad)
{
    if (!M || !t) return sfail(M, PT_ERR_ARG, "NULL argument");
    int rc = load_batch(M, L, B, J, t);
    if (rc) return rc;
    if ((rc = forward(M, B, true))) return rc;
    if ((rc = backward_all(M, B))) return rc;
    SK(cudaGetLastError(), "gradient kernels");
    if (grad) SK(cudaMemcpyAsync(grad, M->grad, sizeof(float) * M->nparams, cudaMemcpyDeviceToHost, M->stream), "download grad");
    float lv = 0.f;
    int terr = 0;
    SK(cudaMemcpyAsync(&lv, M->dloss, sizeof(float), cudaMemcpyDeviceToHost, M->stream), "download loss");
    SK(cudaMemcpyAsync(&terr, M->d_err, sizeof(int), cudaMemcpyDeviceToHost, M->stream), "download status");
    SK(cudaStreamSynchronize(M->stream), "sync grad");
    if (loss) *loss = lv;
    return tc_status(M, terr);
}

int sg_adam(sg_model* M, float lr)
{
    if (!M) return PT_ERR_ARG;
    M->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - (float)std::pow(0.9, (double)M->step), c2 = 1.f - (float)std::pow(0.999, (double)M->step);
    adam_kernel<<<grid_for((size_t)M->nparams), 256, 0, M->stream>>>(M->nparams, M->theta, M->grad, M->mom1, M->mom2,
                                                                        lr, b1, b2, c1, c2, 1e-8f);
    to_bf16_kernel<<<grid_for((size_t)M->nparams), 256, 0, M->stream>>>(M->nparams, M->theta, M->wbf);
    M->launches += 2;
    pack_weights(M);
    SK(cudaGetLastError(), "adam kernels");
    SK(cudaStreamSynchronize(M->stream), "sync adam");
    return PT_OK;
}

int sg_train_step(sg_model* M, int32_t L, int32_t B, const int8_t* J, const float* t, float lr, float* loss)
{
    int rc = sg_grad(M, L, B, J, t, loss, nullptr);
    if (rc) return rc;
    return sg_adam(M, lr);
}

uint64_t sg_launch_count(const sg_model* M) { return M ? M->launches : 0; }

}  // extern "C"
