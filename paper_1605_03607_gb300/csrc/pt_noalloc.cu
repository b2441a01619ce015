// pt_noalloc.cu -- PT-TTS evaluation without any allocation (pt_tts_eval_noalloc).
//
// Some callers cannot allocate device memory when they want an evaluation:
// code that runs inside another framework whose allocator (a caching
// allocator or a memory pool) already owns the device memory, so a fresh
// cudaMalloc fails or fragments it, and latency-critical loops that cannot
// afford the implicit device-wide synchronisation cudaMalloc/cudaFree can
// cause.  This entry point serves them: every device buffer it needs lives in
// one file-scope static __device__ array of fixed size, and every host buffer
// in file-scope static storage.  It calls no cudaMalloc, cudaFree or other
// allocating routine.
//
// Cost and limits: every GPU that loads the library holds the PT_NOALLOC_BYTES
// (4 MiB) array until the process exits.  A problem fits when
//   n_runs * n_temps * 8 L^2 <= 2^21 spin bytes, n_runs * n_temps <= 16384,
//   n_runs <= 1024, and its exchange tables total <= 2^17 entries;
// larger problems are rejected with PT_ERR_ARG.
//
// Every call shares the array, which keeps the previous call's contents; the
// initialisation kernel rewrites every spin, slot map, energy, record and
// counter before use.  Calls whose GPU work overlaps would race on the array
// and on the host staging buffers.  Inside one process that cannot happen
// through this entry point: a call holds a process-wide lock from staging to
// the final stream synchronisation (also on every error path once work is
// queued), so calls from several host threads or streams run one after the
// other.  Two processes each have their own copy of the array.
//
// Set-up: the first call on a device (with that device current) resolves the
// array's device address with cudaGetSymbolAddress and raises the sweep
// kernel's shared-memory limit; make that first call outside any stream
// capture.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/pt.h"
#include "pt_host.h"
#include "pt_internal.h"
#include "pt_kernels.h"

namespace {

using namespace ptg;

constexpr size_t PT_NOALLOC_BYTES = 4u << 20;
constexpr int64_t MAX_SPIN_BYTES = 1 << 21;
constexpr int64_t MAX_REPLICAS = 16384;
constexpr int MAX_RUNS = 1024;
constexpr int64_t MAX_XTHR = 1 << 17;
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_scratch[PT_NOALLOC_BYTES];

// host staging (static: no allocation)
uint32_t h_thr[MAX_TEMPS * KT_MAX];
int64_t h_xoff64[MAX_TEMPS];
int32_t h_xoff[MAX_TEMPS];
float h_xhint[MAX_TEMPS];
uint32_t h_xthr[MAX_XTHR];
uint32_t h_jw[MAX_L * MAX_L * 16];
int16_t h_nbr[MAX_L * MAX_L * 4];
int2 h_items[MAX_RUNS];
Bundle h_bundles[MAX_RUNS];
int32_t h_out[3];

std::mutex g_mu;
unsigned char* g_base[MAX_DEVICES];   // device address of g_scratch per device (set up once)
int g_smem_cap[MAX_DEVICES];

// Failures are reported through pt_last_error(NULL).
int noalloc_fail(int code, const char* msg)
{
    set_global_error(msg);
    return code;
}

// A failed CUDA call: its name and the runtime's message go to
// pt_last_error(NULL).  Once work may be queued on the stream, the stream is
// drained first, so the shared array is idle when the call returns and the
// lock is released.
int noalloc_cuda_fail(const char* what, cudaError_t e, cudaStream_t st, bool queued)
{
    static char msg[256];
    if (queued) cudaStreamSynchronize(st);
    std::snprintf(msg, sizeof(msg), "pt_tts_eval_noalloc: %s: %s", what, cudaGetErrorString(e));
    set_global_error(msg);
    return e == cudaErrorMemoryAllocation ? PT_ERR_OOM : PT_ERR_CUDA;
}

size_t carve(size_t& off, size_t bytes)
{
    const size_t at = off;
    off = (off + bytes + 255) & ~(size_t)255;
    return at;
}

}  // namespace

extern "C" int pt_tts_eval_noalloc(int32_t L, const int8_t* J, int32_t n_edges, const double* betas,
                                   int32_t n_temps, int32_t n_runs, uint32_t seed, uint32_t uid,
                                   int32_t S, int32_t pass_mult, int32_t exchange_every, void* stream,
                                   int32_t* tts, int32_t* n_hit, int32_t* target)
{
    if (!J || !betas || !tts) return noalloc_fail(PT_ERR_ARG, "NULL argument");
    if (L < 1 || L > MAX_L || n_edges != 16 * L * L + 8 * L * (L - 1))
        return noalloc_fail(PT_ERR_ARG, "chimera_L must be in [1, 16] and n_edges = 16 L^2 + 8 L (L-1)");
    if (n_temps < 1 || n_temps > MAX_TEMPS || n_runs < 1 || n_runs > MAX_RUNS)
        return noalloc_fail(PT_ERR_ARG, "n_temps must be in [1, 64] and n_runs in [1, 1024]");
    if (S < 1 || pass_mult < 1 || exchange_every < 0 || (int64_t)S * pass_mult > (1 << 30))
        return noalloc_fail(PT_ERR_ARG, "need S >= 1, pass_mult >= 1, S * pass_mult <= 2^30");
    const int N = 8 * L * L;
    const int64_t reps = (int64_t)n_runs * n_temps;
    if (reps * N > MAX_SPIN_BYTES || reps > MAX_REPLICAS)
        return noalloc_fail(PT_ERR_ARG, "problem exceeds the fixed no-alloc scratch: need n_runs * n_temps * 8 L^2 "
                                        "<= 2^21 and n_runs * n_temps <= 16384");
    for (int e = 0; e < n_edges; ++e)
        if (J[e] < -J_ABS_MAX) return noalloc_fail(PT_ERR_ARG, "coupler outside [-127, 127]");
    const int kmax = coupler_kmax(L, J);
    if (kmax > KT_MAX - 1) return noalloc_fail(PT_ERR_ARG, "a spin's sum of |J| exceeds 127");
    const int kt = table_rows_for(kmax);
    for (int t = 0; t < n_temps; ++t)
        if (!(betas[t] > 0.0) || !std::isfinite(betas[t]) || (t > 0 && !(betas[t] < betas[t - 1])))
            return noalloc_fail(PT_ERR_ARG, "betas must be finite, > 0 and strictly descending");

    std::lock_guard<std::mutex> lock(g_mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES)
        return noalloc_fail(PT_ERR_CUDA, "no usable current CUDA device");
    if (!g_base[dev]) {                                   // once per device, this device current
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) return noalloc_cuda_fail("cudaGetSymbolAddress of the scratch array", e, nullptr, false);
        int cap = 0;
        cudaError_t e2 = sweep_smem_capacity(&cap);
        if (e2 == cudaSuccess) e2 = set_sweep_smem_limit(cap);
        if (e2 != cudaSuccess) return noalloc_cuda_fail("setting the sweep kernel's shared-memory limit", e2, nullptr, false);
        g_smem_cap[dev] = cap;
        g_base[dev] = static_cast<unsigned char*>(p);
    }
    unsigned char* base = g_base[dev];
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    const char* why = "";
    const int64_t nx = fill_tables(n_temps, kt, betas, h_thr, h_xoff64, h_xhint, h_xthr, MAX_XTHR, &why);
    if (nx < 0) return noalloc_fail(PT_ERR_ARG, "exchange tables exceed 2^17 entries (beta gaps too small) or are invalid");
    for (int t = 0; t < n_temps; ++t) h_xoff[t] = (int32_t)h_xoff64[t];
    pack_couplers(L, J, h_jw);
    build_neighbours(L, h_nbr);

    // schedule: about 256 threads per run, a multiple of 32, one run per CTA
    const int L2 = L * L;
    int sp = 256 / L2 > 1 ? 256 / L2 : 1;
    if (sp > n_temps) sp = n_temps;
    while ((sp * L2) % 32 != 0) ++sp;
    const int block = sp * L2;
    const int smem = (int)bundle_smem_bytes(L, n_temps, 1, 0, false, kt);
    if (block > MAX_THREADS || smem > g_smem_cap[dev])
        return noalloc_fail(PT_ERR_ARG, "one run needs more shared memory than a CTA can have");
    for (int r = 0; r < n_runs; ++r) {
        h_items[r] = make_int2(0, r);
        h_bundles[r].inst = 0; h_bundles[r].run0 = r; h_bundles[r].nitems = 1; h_bundles[r].sp = sp;
        h_bundles[r].team = 0;
    }

    // carve the scratch
    size_t off = 0;
    const int npair = n_temps > 1 ? n_temps - 1 : 1;
    const size_t o_spins = carve(off, (size_t)reps * N);
    const size_t o_E = carve(off, 4 * (size_t)reps);
    const size_t o_perm = carve(off, (size_t)reps);
    const size_t o_best = carve(off, 4 * (size_t)n_runs);
    const size_t o_first = carve(off, 4 * (size_t)n_runs);
    const size_t o_macc = carve(off, 8 * (size_t)reps);
    const size_t o_xacc = carve(off, 8 * (size_t)n_runs * npair);
    const size_t o_jw = carve(off, 4 * (size_t)L2 * 16);
    const size_t o_nbr = carve(off, 2 * (size_t)L2 * 4);
    const size_t o_thr = carve(off, 4 * (size_t)n_temps * kt);
    const size_t o_xoff = carve(off, 4 * (size_t)n_temps);
    const size_t o_xhint = carve(off, 4 * (size_t)n_temps);
    const size_t o_xthr = carve(off, 4 * (size_t)(nx > 0 ? nx : 1));
    const size_t o_desc = carve(off, sizeof(InstDesc));
    const size_t o_items = carve(off, sizeof(int2) * (size_t)n_runs);
    const size_t o_bund = carve(off, sizeof(Bundle) * (size_t)n_runs);
    const size_t o_out = carve(off, 16);
    if (off > PT_NOALLOC_BYTES) return noalloc_fail(PT_ERR_ARG, "problem exceeds the 4 MiB no-alloc scratch");

    InstDesc d;
    d.L = L; d.NT = n_temps; d.R = n_runs; d.n_xpairs = n_temps - 1;
    d.seed = seed; d.uid = uid;
    d.kt = kt;
    d.jw = reinterpret_cast<const uint32_t*>(base + o_jw);
    d.nbr = reinterpret_cast<const int16_t*>(base + o_nbr);
    d.thr = reinterpret_cast<const uint32_t*>(base + o_thr);
    d.xoff = reinterpret_cast<const int32_t*>(base + o_xoff);
    d.xthr = reinterpret_cast<const uint32_t*>(base + o_xthr);
    d.xhint = reinterpret_cast<const float*>(base + o_xhint);
    d.spins = reinterpret_cast<int8_t*>(base + o_spins);
    d.E = reinterpret_cast<int32_t*>(base + o_E);
    d.perm = reinterpret_cast<uint8_t*>(base + o_perm);
    d.best = reinterpret_cast<int32_t*>(base + o_best);
    d.first = reinterpret_cast<int32_t*>(base + o_first);
    d.macc = reinterpret_cast<unsigned long long*>(base + o_macc);
    d.xacc = reinterpret_cast<unsigned long long*>(base + o_xacc);
    static InstDesc h_desc;
    h_desc = d;

    cudaError_t ce = cudaSuccess;
    auto up = [&](size_t o, const void* src, size_t bytes) {
        return cudaMemcpyAsync(base + o, src, bytes, cudaMemcpyHostToDevice, st);
    };
    if ((ce = up(o_jw, h_jw, 4 * (size_t)L2 * 16)) != cudaSuccess) return noalloc_cuda_fail("cudaMemcpyAsync (staging upload)", ce, st, true);
    if ((ce = up(o_nbr, h_nbr, 2 * (size_t)L2 * 4)) != cudaSuccess) return noalloc_cuda_fail("cudaMemcpyAsync (staging upload)", ce, st, true);
    if ((ce = up(o_thr, h_thr, 4 * (size_t)n_temps * kt)) != cudaSuccess) return noalloc_cuda_fail("cudaMemcpyAsync (staging upload)", ce, st, true);
    if ((ce = up(o_xoff, h_xoff, 4 * (size_t)n_temps)) != cudaSuccess) return noalloc_cuda_fail("cudaMemcpyAsync (staging upload)", ce, st, true);
    if ((ce = up(o_xhint, h_xhint, 4 * (size_t)n_temps)) != cudaSuccess) return noalloc_cuda_fail("cudaMemcpyAsync (staging upload)", ce, st, true);
    if (nx > 0 && (ce = up(o_xthr, h_xthr, 4 * (size_t)nx)) != cudaSuccess)
        return noalloc_cuda_fail("cudaMemcpyAsync (staging upload)", ce, st, true);
    if ((ce = up(o_desc, &h_desc, sizeof(InstDesc))) != cudaSuccess) return noalloc_cuda_fail("cudaMemcpyAsync (staging upload)", ce, st, true);
    if ((ce = up(o_items, h_items, sizeof(int2) * (size_t)n_runs)) != cudaSuccess) return noalloc_cuda_fail("cudaMemcpyAsync (staging upload)", ce, st, true);
    if ((ce = up(o_bund, h_bundles, sizeof(Bundle) * (size_t)n_runs)) != cudaSuccess) return noalloc_cuda_fail("cudaMemcpyAsync (staging upload)", ce, st, true);

    const InstDesc* dd = reinterpret_cast<const InstDesc*>(base + o_desc);
    const int2* di = reinterpret_cast<const int2*>(base + o_items);
    const Bundle* db = reinterpret_cast<const Bundle*>(base + o_bund);
    int32_t* dout = reinterpret_cast<int32_t*>(base + o_out);
    // fresh runs: the init kernel draws every spin and zeroes every counter,
    // the energy kernel sets energies and records
    if ((ce = launch_init(dd, di, n_runs, true, st)) != cudaSuccess) return noalloc_cuda_fail("init kernel", ce, st, true);
    if ((ce = launch_energy(dd, di, n_runs, 0, st)) != cudaSuccess) return noalloc_cuda_fail("energy kernel", ce, st, true);
    const int64_t total = (int64_t)S * pass_mult;
    for (int64_t done = 0; done < total;) {
        const int chunk = (int)(total - done < 4096 ? total - done : 4096);
        if ((ce = launch_sweeps(dd, db, n_runs, n_runs, block, smem, (uint32_t)done, chunk, exchange_every, 0,
                                nullptr, st)) != cudaSuccess)
            return noalloc_cuda_fail("sweep kernel", ce, st, true);
        done += chunk;
    }
    if ((ce = launch_tts(dd, 1, PT_TARGET_BEST, S, dout, st)) != cudaSuccess) return noalloc_cuda_fail("TTS kernel", ce, st, true);
    if ((ce = cudaMemcpyAsync(h_out, dout, sizeof(h_out), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return noalloc_cuda_fail("cudaMemcpyAsync (result download)", ce, st, true);
    if ((ce = cudaStreamSynchronize(st)) != cudaSuccess) return noalloc_cuda_fail("cudaStreamSynchronize", ce, st, false);
    *tts = h_out[0];
    if (n_hit) *n_hit = h_out[1];
    if (target) *target = h_out[2];
    return PT_OK;
}
