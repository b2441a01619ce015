// int_peak.cu -- integer-issue microbenchmark (pt_int_issue_rate).
//
// The sweep kernel does no dense contraction and keeps its replicas in shared
// memory, so its ceiling is the rate at which the SMs issue 32-bit integer
// instructions.  The roofline peak is derived from unit counts and the clock
// (SMs x 4 sub-partitions x 32 lanes x f).  This kernel measures what the
// hardware sustains for the instruction kinds the sweep is made of, so the
// derived peak can be read against a measured one:
//
//   kind 0  LOP3:  three-input logic (xor of three words)
//   kind 1  IMAD:  32-bit multiply-add
//   kind 2  LOP3 and IMAD interleaved one to one
//   kind 3  DP4A:  four-way int8 dot product with accumulate (the local fields)
//   kind 4  Philox4x32-10 rounds: two states sharing one key schedule, so an
//           iteration is four widening 32x32->64 multiplies, four three-input
//           xors and two key adds (10 operations)
//
// Every thread runs independent dependency chains (8 words, or 2 Philox
// states), so issue, not latency, limits the rate.  Each operation is one
// inline PTX instruction whose result feeds the next iteration, and every
// thread stores its final state, so nothing can be folded away.  The grid is
// 8 CTAs of 256 threads per SM (64 warps per SM, 16 per sub-partition).
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/pt.h"
#include "pt_internal.h"

namespace {

constexpr int IP_THREADS = 256;
constexpr int IP_CTAS_PER_SM = 8;
constexpr int IP_MAX_ITERS = 1 << 22;
constexpr int IP_MAX_REPS = 1000;

__device__ __forceinline__ uint32_t op_lop3(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

__device__ __forceinline__ uint32_t op_imad(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

__device__ __forceinline__ uint32_t op_dp4a(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("dp4a.s32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

__device__ __forceinline__ void op_mulwide(uint32_t a, uint32_t m, uint32_t& hi, uint32_t& lo)
{
    uint64_t p;
    asm("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(a), "r"(m));
    hi = (uint32_t)(p >> 32);
    lo = (uint32_t)p;
}

__device__ __forceinline__ uint32_t op_add(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("add.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

template <int KIND>
__global__ void __launch_bounds__(IP_THREADS, IP_CTAS_PER_SM)
int_issue_kernel(int iters, uint32_t* __restrict__ out)
{
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    if constexpr (KIND == 4) {
        // two Philox states per thread sharing one (per-thread) key schedule
        uint32_t x0 = tid, x1 = ~tid, x2 = tid * 3u, x3 = tid ^ 0x5bd1e995u;
        uint32_t y0 = tid + 1u, y1 = tid * 7u, y2 = ~tid * 5u, y3 = tid ^ 0x27d4eb2fu;
        uint32_t k0 = tid * 11u, k1 = tid * 13u;
        const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u, w0 = 0x9E3779B9u, w1 = 0xBB67AE85u;
        for (int i = 0; i < iters; ++i) {
            uint32_t h0, l0, h1, l1;
            op_mulwide(x0, m0, h0, l0);
            op_mulwide(x2, m1, h1, l1);
            const uint32_t nx0 = op_lop3(h1, x1, k0), nx2 = op_lop3(h0, x3, k1);
            x1 = l1; x3 = l0; x0 = nx0; x2 = nx2;
            op_mulwide(y0, m0, h0, l0);
            op_mulwide(y2, m1, h1, l1);
            const uint32_t ny0 = op_lop3(h1, y1, k1), ny2 = op_lop3(h0, y3, k0);
            y1 = l1; y3 = l0; y0 = ny0; y2 = ny2;
            k0 = op_add(k0, w0);
            k1 = op_add(k1, w1);
        }
        out[tid] = x0 ^ x1 ^ x2 ^ x3 ^ y0 ^ y1 ^ y2 ^ y3;
    } else {
        uint32_t a[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) a[c] = tid * (2u * c + 1u) + 0x9E3779B9u * c;
        for (int i = 0; i < iters; ++i) {
            const uint32_t x = (uint32_t)i;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const uint32_t b = a[(c + 1) & 7];
                if (KIND == 0) a[c] = op_lop3(a[c], b, x);
                else if (KIND == 1) a[c] = op_imad(a[c], b, x);
                else if (KIND == 2) a[c] = (c & 1) ? op_imad(a[c], b, x) : op_lop3(a[c], b, x);
                else a[c] = op_dp4a(a[c], b, x);
            }
        }
        uint32_t r = 0;
#pragma unroll
        for (int c = 0; c < 8; ++c) r ^= a[c];
        out[tid] = r;
    }
}

// Operations one thread performs per loop iteration.
double ops_per_iter(int kind)
{
    // kind 4: 2 states x (2 multiplies + 2 xors) + 2 key adds
    return kind == 4 ? 10.0 : 8.0;
}

cudaError_t launch_kind(int kind, int grid, int iters, uint32_t* out, cudaStream_t st)
{
    switch (kind) {
    case 0: int_issue_kernel<0><<<grid, IP_THREADS, 0, st>>>(iters, out); break;
    case 1: int_issue_kernel<1><<<grid, IP_THREADS, 0, st>>>(iters, out); break;
    case 2: int_issue_kernel<2><<<grid, IP_THREADS, 0, st>>>(iters, out); break;
    case 3: int_issue_kernel<3><<<grid, IP_THREADS, 0, st>>>(iters, out); break;
    default: int_issue_kernel<4><<<grid, IP_THREADS, 0, st>>>(iters, out); break;
    }
    return cudaGetLastError();
}

int ip_fail(int code, const char* msg)
{
    ptg::set_global_error(msg);
    return code;
}

}  // namespace

extern "C" int pt_int_issue_rate(int32_t kind, int32_t iters, int32_t reps, double* ops_per_s,
                                 double* ms_per_launch, void* stream)
{
    if (!ops_per_s) return ip_fail(PT_ERR_ARG, "ops_per_s is NULL");
    if (kind < 0 || kind > 4) return ip_fail(PT_ERR_ARG, "kind must be in [0, 4]");
    if (iters < 1 || iters > IP_MAX_ITERS) return ip_fail(PT_ERR_ARG, "iters must be in [1, 2^22]");
    if (reps < 1 || reps > IP_MAX_REPS) return ip_fail(PT_ERR_ARG, "reps must be in [1, 1000]");
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return ip_fail(PT_ERR_CUDA, "no usable current CUDA device");
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int grid = sms * IP_CTAS_PER_SM;
    uint32_t* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = PT_OK;
    float ms = 0.0f;
    if (cudaMalloc(&out, (size_t)grid * IP_THREADS * sizeof(uint32_t)) != cudaSuccess)
        return ip_fail(PT_ERR_OOM, "cudaMalloc of the output words failed");
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = ip_fail(PT_ERR_CUDA, "cudaEventCreate failed");
        goto done;
    }
    if (launch_kind(kind, grid, iters, out, st) != cudaSuccess) {      // warm-up
        rc = ip_fail(PT_ERR_CUDA, "microbenchmark launch failed");
        goto done;
    }
    cudaEventRecord(e0, st);
    for (int r = 0; r < reps; ++r) {
        if (launch_kind(kind, grid, iters, out, st) != cudaSuccess) {
            rc = ip_fail(PT_ERR_CUDA, "microbenchmark launch failed");
            goto done;
        }
    }
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        rc = ip_fail(PT_ERR_CUDA, "microbenchmark timing failed");
        goto done;
    }
    {
        const double per_launch = (double)ms / reps;
        const double ops = (double)grid * IP_THREADS * (double)iters * ops_per_iter(kind);
        *ops_per_s = per_launch > 0.0 ? ops / (per_launch * 1e-3) : 0.0;
        if (ms_per_launch) *ms_per_launch = per_launch;
    }
done:
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    return rc;
}
