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
// node or edge row) run on tensor cores (mma.sync m16n8k16 BF16).  Gradients
// are FP32 buffers; master weights and Adam moments are FP32.
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

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
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

// ------------------------------------------------------------ forward GEMM
// Z = W X + bias for 16 rows per warp, W [64][128] BF16 staged in shared
// memory.  EPI 0 (messages): Z -> Zout (BF16), relu(Z) -> Rout (FP32).
// EPI 1 (residual): Z -> Zout, Yout = P0 row + relu(Z) (BF16).
template <int EPI>
__global__ void __launch_bounds__(256) lin_fwd_kernel(int rows, RowSrc src, const bf16* __restrict__ W,
                                                      const float* __restrict__ bias, bf16* __restrict__ Zout,
                                                      float* __restrict__ Rout, bf16* __restrict__ Yout)
{
    __shared__ uint32_t Ws[HD][KIN / 2 + 4];
    for (int i = threadIdx.x; i < HD * KIN / 2; i += blockDim.x)
        Ws[i / (KIN / 2)][i % (KIN / 2)] = reinterpret_cast<const uint32_t*>(W)[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int warps = blockDim.x >> 5;
    const int ntiles = (rows + 15) / 16;
    for (int tile = blockIdx.x * warps + (threadIdx.x >> 5); tile < ntiles; tile += gridDim.x * warps) {
        const int ra = tile * 16 + g, rb = ra + 8;
        const bool va = ra < rows, vb = rb < rows;
        const uint32_t* pa0 = va ? src.half(ra, 0) : nullptr;
        const uint32_t* pa1 = va ? src.half(ra, 1) : nullptr;
        const uint32_t* pb0 = vb ? src.half(rb, 0) : nullptr;
        const uint32_t* pb1 = vb ? src.half(rb, 1) : nullptr;
        float acc[8][4];
#pragma unroll
        for (int n = 0; n < 8; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
#pragma unroll
        for (int ks = 0; ks < 8; ++ks) {
            const int cw = (ks & 3) * 8 + t;          // u32 index inside the 64-wide half
            const uint32_t* sa = ks < 4 ? pa0 : pa1;
            const uint32_t* sb = ks < 4 ? pb0 : pb1;
            const uint32_t a0 = va ? sa[cw] : 0u, a2 = va ? sa[cw + 4] : 0u;
            const uint32_t a1 = vb ? sb[cw] : 0u, a3 = vb ? sb[cw + 4] : 0u;
#pragma unroll
            for (int n = 0; n < 8; ++n)
                mma_bf16(acc[n], a0, a1, a2, a3, Ws[n * 8 + g][ks * 8 + t], Ws[n * 8 + g][ks * 8 + 4 + t]);
        }
#pragma unroll
        for (int n = 0; n < 8; ++n) {
            const int c = n * 8 + 2 * t;
            const float b0 = bias[c], b1 = bias[c + 1];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = h ? rb : ra;
                if (!(h ? vb : va)) continue;
                const float z0 = acc[n][2 * h] + b0, z1 = acc[n][2 * h + 1] + b1;
                reinterpret_cast<uint32_t*>(Zout + (size_t)r * HD)[c / 2] = pack_bf2(z0, z1);
                if (EPI == 0) {
                    reinterpret_cast<float2*>(Rout + (size_t)r * HD)[c / 2] = make_float2(fmaxf(z0, 0.f), fmaxf(z1, 0.f));
                } else {
                    const float2 base = unpack_bf2((h ? pb0 : pa0)[c / 2]);
                    reinterpret_cast<uint32_t*>(Yout + (size_t)r * HD)[c / 2] =
                        pack_bf2(base.x + fmaxf(z0, 0.f), base.y + fmaxf(z1, 0.f));
                }
            }
        }
    }
}

__device__ __forceinline__ void ldsm_x4(uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3, const void* p)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(a));
}

// ------------------------------------------------ backward: dX = dZ . W
// dZ [rows][64] BF16, each warp's 16-row tile staged in shared memory with
// 16-byte loads and read by ldmatrix; W^T staged as [128][64].  Launched
// with 256 threads (8 warps).  EPI 0: dX [rows][128] FP32.
// EPI 1 (the node and edge updates, whose input halves have separate
// gradients): out0 = base + dX[:, :64] (base may be out0 or NULL) and
// out1 = dX[:, 64:], both [rows][64] FP32, without materialising dX.
template <int EPI>
__global__ void __launch_bounds__(256) lin_bwd_input_kernel(int rows, const bf16* __restrict__ dZ,
                                                            const bf16* __restrict__ W, float* __restrict__ dX,
                                                            const float* base, float* out0, float* __restrict__ out1)
{
    __shared__ uint32_t WT[KIN][HD / 2 + 4];
    for (int i = threadIdx.x; i < KIN * HD / 2; i += blockDim.x) {
        const int in = i / (HD / 2), op = i % (HD / 2);        // pair of outputs 2op, 2op+1
        const float w0 = __bfloat162float(W[(2 * op) * KIN + in]);
        const float w1 = __bfloat162float(W[(2 * op + 1) * KIN + in]);
        __nv_bfloat162 v = __floats2bfloat162_rn(w0, w1);
        WT[in][op] = *reinterpret_cast<uint32_t*>(&v);
    }
    __syncthreads();
    __shared__ __align__(16) bf16 Zs[8][16][HD + 8];
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3, w = threadIdx.x >> 5;
    const int lr = lane & 7, lq = lane >> 3;
    bf16 (*Zt)[HD + 8] = Zs[w];
    const int warps = blockDim.x >> 5;
    const int ntiles = (rows + 15) / 16;
    for (int tile = blockIdx.x * warps + w; tile < ntiles; tile += gridDim.x * warps) {
        const int ra = tile * 16 + g, rb = ra + 8;
        const bool va = ra < rows, vb = rb < rows;
#pragma unroll
        for (int j = 0; j < 4; ++j) {                 // 16 rows x 8 16-byte words of dZ
            const int i = lane + 32 * j, rr = i >> 3, q = i & 7, r = tile * 16 + rr;
            const uint4 v = r < rows ? reinterpret_cast<const uint4*>(dZ + (size_t)r * HD)[q] : make_uint4(0u, 0u, 0u, 0u);
            *reinterpret_cast<uint4*>(&Zt[rr][q * 8]) = v;
        }
        __syncwarp();
        float acc[16][4];
#pragma unroll
        for (int n = 0; n < 16; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
            uint32_t a0, a1, a2, a3;
            ldsm_x4(a0, a1, a2, a3, &Zt[(lq & 1) * 8 + lr][ks * 16 + (lq >> 1) * 8]);
#pragma unroll
            for (int n = 0; n < 16; ++n)
                mma_bf16(acc[n], a0, a1, a2, a3, WT[n * 8 + g][ks * 8 + t], WT[n * 8 + g][ks * 8 + 4 + t]);
        }
        __syncwarp();                                 // the tile is read before it is restaged
#pragma unroll
        for (int n = 0; n < 16; ++n) {
            const int c = n * 8 + 2 * t;
            if (EPI == 0) {
                if (va) reinterpret_cast<float2*>(dX + (size_t)ra * KIN)[c / 2] = make_float2(acc[n][0], acc[n][1]);
                if (vb) reinterpret_cast<float2*>(dX + (size_t)rb * KIN)[c / 2] = make_float2(acc[n][2], acc[n][3]);
            } else if (n < 8) {
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const int r = hh ? rb : ra;
                    if (!(hh ? vb : va)) continue;
                    float2 v = make_float2(acc[n][2 * hh], acc[n][2 * hh + 1]);
                    if (base) {
                        const float2 b = reinterpret_cast<const float2*>(base + (size_t)r * HD)[c / 2];
                        v.x = b.x + v.x;
                        v.y = b.y + v.y;
                    }
                    reinterpret_cast<float2*>(out0 + (size_t)r * HD)[c / 2] = v;
                }
            } else {
                if (va) reinterpret_cast<float2*>(out1 + (size_t)ra * HD)[c / 2 - HD / 2] = make_float2(acc[n][0], acc[n][1]);
                if (vb) reinterpret_cast<float2*>(out1 + (size_t)rb * HD)[c / 2 - HD / 2] = make_float2(acc[n][2], acc[n][3]);
            }
        }
    }
}

// ------------------------------- backward: dW = dZ^T . X, db = column sums of dZ
// Persistent blocks take 64-row chunks c = blockIdx.x, c += gridDim.x.  A
// chunk is staged row-major with 16-byte loads (dZ [64][64], X [64][128] from
// its two gathered halves), the next chunk's loads are issued into registers
// before the current chunk's MMAs, and ldmatrix.trans transposes the 8x8
// sub-tiles on their way into the mma.sync fragments (A = dZ^T, B = X).
// Warp w accumulates output rows 16*(w/2)..+16 and columns 64*(w%2)..+64;
// the even warps also sum their rows of dZ (one extra MMA against ones).
// Each block writes its partial [64][128] + [64] to `part`, and
// lin_wgrad_reduce adds all blocks' partials into dW and db in a fixed order.
constexpr int WCH = 64;                  // rows per chunk
constexpr int ZP = HD + 8;               // shared row pitches (bf16): 16 bytes of padding
constexpr int XP = KIN + 8;              // make every ldmatrix phase conflict-free
constexpr int WPART = HD * KIN + HD;     // floats of one block's partial

__device__ __forceinline__ void ldsm_x4_trans(uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3, const void* p)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(a));
}

struct WChunk {                          // one thread's share of a chunk: 2 + 4 16-byte words
    uint4 z[2], x[4];
};

__device__ __forceinline__ void wgrad_load(WChunk& v, int rows, int r0, const bf16* __restrict__ dZ,
                                           const RowSrc& src)
{
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int i = threadIdx.x + j * 256, rr = i >> 3, q = i & 7, r = r0 + rr;
        v.z[j] = r < rows ? reinterpret_cast<const uint4*>(dZ + (size_t)r * HD)[q] : make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int i = threadIdx.x + j * 256, rr = i >> 4, seg = i & 15, r = r0 + rr;
        v.x[j] = r < rows ? reinterpret_cast<const uint4*>(src.half(r, seg >> 3))[seg & 7] : make_uint4(0u, 0u, 0u, 0u);
    }
}

__global__ void __launch_bounds__(256, 2) lin_wgrad_kernel(int rows, const bf16* __restrict__ dZ, RowSrc src,
                                                           float* __restrict__ part)
{
    __shared__ __align__(16) bf16 Zs[WCH][ZP];
    __shared__ __align__(16) bf16 Xs[WCH][XP];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
    const int lr = lane & 7, lq = lane >> 3;          // ldmatrix: row inside an 8x8 tile, tile index
    const int mrow = (w >> 1) * 16, ncol = (w & 1) * 64;
    const uint32_t ones = 0x3F803F80u;                // two bf16 1.0
    float acc[8][4], accb[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int n = 0; n < 8; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
    const int nchunks = (rows + WCH - 1) / WCH;
    WChunk v;
    int c = blockIdx.x;
    if (c < nchunks) wgrad_load(v, rows, c * WCH, dZ, src);
    for (; c < nchunks; c += gridDim.x) {
        __syncthreads();                              // the previous chunk's MMAs are done
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int i = threadIdx.x + j * 256;
            *reinterpret_cast<uint4*>(&Zs[i >> 3][(i & 7) * 8]) = v.z[j];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int i = threadIdx.x + j * 256;
            *reinterpret_cast<uint4*>(&Xs[i >> 4][(i & 15) * 8]) = v.x[j];
        }
        __syncthreads();
        if (c + (int)gridDim.x < nchunks) wgrad_load(v, rows, (c + gridDim.x) * WCH, dZ, src);
#pragma unroll
        for (int ks = 0; ks < WCH / 16; ++ks) {
            const int k0 = ks * 16;
            uint32_t a0, a1, a2, a3;                  // (m0-7,k0-7) (m8-15,k0-7) (m0-7,k8-15) (m8-15,k8-15)
            ldsm_x4_trans(a0, a1, a2, a3, &Zs[k0 + (lq >> 1) * 8 + lr][mrow + (lq & 1) * 8]);
            if ((w & 1) == 0) mma_bf16(accb, a0, a1, a2, a3, ones, ones);
#pragma unroll
            for (int np = 0; np < 4; ++np) {          // n-tiles n0 and n0 + 8
                const int n0 = ncol + np * 16;
                uint32_t b0, b1, b2, b3;              // (k0-7,n0) (k8-15,n0) (k0-7,n0+8) (k8-15,n0+8)
                ldsm_x4_trans(b0, b1, b2, b3, &Xs[k0 + (lq & 1) * 8 + lr][n0 + (lq >> 1) * 8]);
                mma_bf16(acc[2 * np], a0, a1, a2, a3, b0, b1);
                mma_bf16(acc[2 * np + 1], a0, a1, a2, a3, b2, b3);
            }
        }
    }
    float* P = part + (size_t)blockIdx.x * WPART;
#pragma unroll
    for (int n = 0; n < 8; ++n) {
        const int col = ncol + n * 8 + 2 * t;
        *reinterpret_cast<float2*>(&P[(mrow + g) * KIN + col]) = make_float2(acc[n][0], acc[n][1]);
        *reinterpret_cast<float2*>(&P[(mrow + g + 8) * KIN + col]) = make_float2(acc[n][2], acc[n][3]);
    }
    if ((w & 1) == 0 && t == 0) {                     // every column of the ones tile is the row sum
        P[HD * KIN + mrow + g] = accb[0];
        P[HD * KIN + mrow + g + 8] = accb[2];
    }
}

// dW += sum over blocks of the partials (and db likewise), blocks in order.
__global__ void lin_wgrad_reduce(int nblocks, const float* __restrict__ part, float* __restrict__ dW,
                                 float* __restrict__ db)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= WPART) return;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    int b = 0;
    for (; b + 4 <= nblocks; b += 4) {
        s0 += part[(size_t)b * WPART + i];
        s1 += part[(size_t)(b + 1) * WPART + i];
        s2 += part[(size_t)(b + 2) * WPART + i];
        s3 += part[(size_t)(b + 3) * WPART + i];
    }
    for (; b < nblocks; ++b) s0 += part[(size_t)b * WPART + i];
    const float s = (s0 + s1) + (s2 + s3);
    if (i < HD * KIN) dW[i] += s;
    else db[i - HD * KIN] += s;
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

// de[b][e] += dXm[b][2e][64..] + dXm[b][2e+1][64..]
__global__ void edge_from_messages_kernel(int B, int E, const float* __restrict__ dXm, float* de)
{
    const size_t total = (size_t)B * E * HD;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t be = i / HD;
        const int c = (int)(i % HD);
        const int b = (int)(be / E), e = (int)(be % E);
        const size_t r0 = (size_t)b * 2 * E + 2 * e;
        de[i] += dXm[r0 * KIN + HD + c] + dXm[(r0 + 1) * KIN + HD + c];
    }
}

// readout forward + loss gradient (one block per graph, HD threads)
__global__ void readout_kernel(int N, const bf16* __restrict__ h, const float* __restrict__ W1, const float* __restrict__ b1,
                               const float* __restrict__ w2, const float* __restrict__ b2, float* y, float* gbuf,
                               float* zbuf, const float* __restrict__ target, float inv_B, float* loss,
                               float* dh, float* dW1, float* db1, float* dw2, float* db2)
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
    if (c == 0) {
        atomicAdd(loss, (yb - target[b]) * (yb - target[b]) * inv_B);
        atomicAdd(db2, dy);
    }
    atomicAdd(&dw2[c], dy * as[c]);
    dz[c] = z > 0.f ? dy * w2[c] : 0.f;
    atomicAdd(&db1[c], dz[c]);
    __syncthreads();
    for (int k = 0; k < HD; ++k) atomicAdd(&dW1[c * HD + k], dz[c] * gs[k]);
    float dg = 0.f;
    for (int o = 0; o < HD; ++o) dg += dz[o] * W1[o * HD + c];
    dg /= (float)N;
    for (int n = 0; n < N; ++n) dh[((size_t)b * N + n) * HD + c] = dg;
}

// embedding gradients: per-block partial sums in shared memory, then atomics
__global__ void embed_bwd_kernel(int B, int N, int E, const int* __restrict__ u, const int8_t* __restrict__ J,
                                 const float* __restrict__ dh, const float* __restrict__ de, float* dX, float* dJt)
{
    __shared__ float sx[2 * HD], sj[6 * HD];
    for (int i = threadIdx.x; i < 2 * HD; i += blockDim.x) sx[i] = 0.f;
    for (int i = threadIdx.x; i < 6 * HD; i += blockDim.x) sj[i] = 0.f;
    __syncthreads();
    const int c = threadIdx.x % HD, lanes = blockDim.x / HD;
    const size_t nrows = (size_t)B * (N + E);
    for (size_t row = blockIdx.x * (size_t)lanes + threadIdx.x / HD; row < nrows; row += (size_t)gridDim.x * lanes) {
        if (row < (size_t)B * N) {
            atomicAdd(&sx[u[row % N] * HD + c], dh[row * HD + c]);
        } else {
            const size_t re = row - (size_t)B * N;
            const int j = J[re];
            atomicAdd(&sj[(j < 0 ? j + 3 : j + 2) * HD + c], de[re * HD + c]);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * HD; i += blockDim.x) atomicAdd(&dX[i], sx[i]);
    for (int i = threadIdx.x; i < 6 * HD; i += blockDim.x) atomicAdd(&dJt[i], sj[i]);
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
    std::vector<bf16*> h, e, m, s, zm, zu, ze;
    float *R = nullptr, *dX = nullptr, *dh = nullptr, *dh2 = nullptr, *de = nullptr, *dm = nullptr, *ds = nullptr;
    bf16* dZ = nullptr;
    float* wpart = nullptr;       // weight-gradient partials, one WPART block per persistent CTA
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
    float** fl[] = {&M->d_t, &M->d_y, &M->d_g, &M->d_z, &M->R, &M->dX, &M->dh, &M->dh2, &M->de, &M->dm, &M->ds};
    for (float** p : fl) { cudaFree(*p); *p = nullptr; }
    cudaFree(M->dZ); M->dZ = nullptr;
    cudaFree(M->wpart); M->wpart = nullptr;
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
    SK(salloc(&M->dX, nM * KIN), "cudaMalloc dX");
    SK(salloc(&M->dZ, nM * HD), "cudaMalloc dZ");
    {
        int dev = 0, sms = 0;
        SK(cudaGetDevice(&dev), "cudaGetDevice");
        SK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device attribute");
        M->wblocks = 2 * sms;                 // two resident CTAs per SM (launch bounds)
        SK(salloc(&M->wpart, (size_t)M->wblocks * WPART), "cudaMalloc wpart");
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

int lin_grid(int rows)
{
    const int tiles = (rows + 15) / 16;
    const int g = (tiles + 7) / 8;
    return g > 4096 ? 4096 : (g < 1 ? 1 : g);
}

// dW += dZ^T X, db += column sums of dZ over `rows` rows (two launches).
void lin_wgrad(sg_model* M, int rows, const RowSrc& src, float* dW, float* db)
{
    const int nchunks = (rows + WCH - 1) / WCH;
    const int grid = nchunks < M->wblocks ? (nchunks > 0 ? nchunks : 1) : M->wblocks;
    lin_wgrad_kernel<<<grid, 256, 0, M->stream>>>(rows, M->dZ, src, M->wpart);
    lin_wgrad_reduce<<<(WPART + 255) / 256, 256, 0, M->stream>>>(grid, M->wpart, dW, db);
}

int forward(sg_model* M, int B, bool train)
{
    const int N = M->N, E = M->E;
    const bf16* W = M->wbf;
    cudaStream_t st = M->stream;
    embed_kernel<<<grid_for((size_t)B * (N + E) * HD), 256, 0, st>>>(B, N, E, M->d_u, M->d_J, M->theta + M->oX,
                                                                       M->theta + M->oJ, M->h[0], M->e[0]);
    M->launches++;
    for (int l = 0; l < M->layers; ++l) {
        // messages: row 2e / 2e+1 of every graph: [h[src] | e[edge]]
        const RowSrc ms = rows_of(M->h[l], M->d_src, N, M->e[l], M->d_eid, E, 2 * E);
        lin_fwd_kernel<0><<<lin_grid(B * 2 * E), 256, 0, st>>>(B * 2 * E, ms, W + M->oWm[l], M->theta + M->obm[l],
                                                              M->zm[l], M->R, nullptr);
        aggregate_kernel<<<grid_for((size_t)B * N * HD / 2), 256, 0, st>>>(B, N, E, M->d_in_rows, M->R, M->m[l]);
        const RowSrc ns = rows_of(M->h[l], M->d_iden, N, M->m[l], M->d_iden, N, N);
        lin_fwd_kernel<1><<<lin_grid(B * N), 256, 0, st>>>(B * N, ns, W + M->oWu[l], M->theta + M->obu[l], M->zu[l],
                                                          nullptr, M->h[l + 1]);
        endpoint_sum_kernel<<<grid_for((size_t)B * E * HD / 2), 256, 0, st>>>(B, N, E, M->d_ei, M->d_ej, M->h[l + 1], M->s[l]);
        const RowSrc es = rows_of(M->e[l], M->d_iden, E, M->s[l], M->d_iden, E, E);
        lin_fwd_kernel<1><<<lin_grid(B * E), 256, 0, st>>>(B * E, es, W + M->oWe[l], M->theta + M->obe[l], M->ze[l],
                                                          nullptr, M->e[l + 1]);
        M->launches += 5;
    }
    (void)train;
    return PT_OK;
}

// Gradient of the mean squared error into M->grad (zeroed first); loss into M->dloss.
int backward_all(sg_model* M, int B)
{
    const int N = M->N, E = M->E;
    const bf16* W = M->wbf;
    cudaStream_t st = M->stream;
    float* G = M->grad;
    SK(cudaMemsetAsync(G, 0, sizeof(float) * M->nparams, st), "zero grad");
    SK(cudaMemsetAsync(M->dloss, 0, sizeof(float), st), "zero loss");
    SK(cudaMemsetAsync(M->de, 0, sizeof(float) * (size_t)B * E * HD, st), "zero de");
    readout_kernel<<<B, HD, 0, st>>>(N, M->h[M->layers], M->theta + M->oW1, M->theta + M->ob1, M->theta + M->ow2,
                                     M->theta + M->ob2, M->d_y, M->d_g, M->d_z, M->d_t, 1.f / (float)B, M->dloss,
                                     M->dh, G + M->oW1, G + M->ob1, G + M->ow2, G + M->ob2);
    M->launches++;
    const size_t nN = (size_t)B * N, nE = (size_t)B * E;
    for (int l = M->layers - 1; l >= 0; --l) {
        // edge update: e' = e + relu(ze), ze = We [e | s] + be
        relu_mask_kernel<<<grid_for(nE * HD / 2), 256, 0, st>>>(B * E, M->de, nullptr, 1, 1, M->ze[l], M->dZ);
        // de += dX[:, :64] (into e), ds = dX[:, 64:]
        lin_bwd_input_kernel<1><<<lin_grid(B * E), 256, 0, st>>>(B * E, M->dZ, W + M->oWe[l], nullptr, M->de,
                                                                 M->de, M->ds);
        const RowSrc es = rows_of(M->e[l], M->d_iden, E, M->s[l], M->d_iden, E, E);
        lin_wgrad(M, B * E, es, G + M->oWe[l], G + M->obe[l]);
        SK(cudaMemcpyAsync(M->dh2, M->dh, sizeof(float) * nN * HD, cudaMemcpyDeviceToDevice, st), "copy dh");
        gather_add_kernel<<<grid_for(nN * HD), 256, 0, st>>>(B, N, E, M->d_inc, M->ds, HD, 0, M->dh2);
        // node update: h' = h + relu(zu), zu = Wu [h | m] + bu
        relu_mask_kernel<<<grid_for(nN * HD / 2), 256, 0, st>>>(B * N, M->dh2, nullptr, 1, 1, M->zu[l], M->dZ);
        // dh = dh2 + dX[:, :64] (into h), dm = dX[:, 64:]
        lin_bwd_input_kernel<1><<<lin_grid(B * N), 256, 0, st>>>(B * N, M->dZ, W + M->oWu[l], nullptr, M->dh2,
                                                                 M->dh, M->dm);
        const RowSrc ns = rows_of(M->h[l], M->d_iden, N, M->m[l], M->d_iden, N, N);
        lin_wgrad(M, B * N, ns, G + M->oWu[l], G + M->obu[l]);
        // messages: m_i = sum relu(zm) over rows into i
        relu_mask_kernel<<<grid_for(nE * 2 * HD / 2), 256, 0, st>>>(B * 2 * E, M->dm, M->d_tgt, 2 * E, N, M->zm[l], M->dZ);
        lin_bwd_input_kernel<0><<<lin_grid(B * 2 * E), 256, 0, st>>>(B * 2 * E, M->dZ, W + M->oWm[l], M->dX,
                                                                     nullptr, nullptr, nullptr);
        const RowSrc ms = rows_of(M->h[l], M->d_src, N, M->e[l], M->d_eid, E, 2 * E);
        lin_wgrad(M, B * 2 * E, ms, G + M->oWm[l], G + M->obm[l]);
        gather_add_kernel<<<grid_for(nN * HD), 256, 0, st>>>(B, N, 2 * E, M->d_out_rows, M->dX, KIN, 0, M->dh);
        edge_from_messages_kernel<<<grid_for(nE * HD), 256, 0, st>>>(B, E, M->dX, M->de);
        M->launches += 15;
    }
    embed_bwd_kernel<<<256, 256, 0, st>>>(B, N, E, M->d_u, M->d_J, M->dh, M->de, G + M->oX, G + M->oJ);
    M->launches++;
    return PT_OK;
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
    *out = M;
    return PT_OK;
}

void sg_destroy(sg_model* M)
{
    if (!M) return;
    if (M->stream) cudaStreamSynchronize(M->stream);
    free_graph(M);
    cudaFree(M->theta); cudaFree(M->grad); cudaFree(M->mom1); cudaFree(M->mom2); cudaFree(M->wbf); cudaFree(M->dloss);
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
                                            0.f, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
    M->launches++;
    SK(cudaGetLastError(), "forward kernels");
    SK(cudaMemcpyAsync(y, M->d_y, sizeof(float) * B, cudaMemcpyDeviceToHost, M->stream), "download y");
    SK(cudaStreamSynchronize(M->stream), "sync forward");
    return PT_OK;
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
    SK(cudaMemcpyAsync(&lv, M->dloss, sizeof(float), cudaMemcpyDeviceToHost, M->stream), "download loss");
    SK(cudaStreamSynchronize(M->stream), "sync grad");
    if (loss) *loss = lv;
    return PT_OK;
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
