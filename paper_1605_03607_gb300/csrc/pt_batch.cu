// pt_batch.cu -- batched PT of many instances of uneven size and temperature
// count in one graph replay (C ABI: pt_batch_* in pt.h).
//
// Every (instance, run) pair is an independent PT run (Sec. II).  Instances
// are grouped by Chimera size, and each size group has its own thread mapping,
// schedule, CTA size and persistent grid.  The host packs a group's runs into
// CTA bundles (a few runs of one instance), orders them by cost (longest
// first), and the group's persistent kernel pulls bundles from its own atomic
// counter until none is left.  The counter reset and one persistent launch per
// group, as concurrent graph branches (largest work at the highest priority, so
// the smaller groups fill its tail), are captured once in a CUDA graph; each
// pt_batch_run replays it with the sweep counter patched into the kernel
// nodes.  Schedules come from pt_batch_autotune and never change results.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <map>
#include <numeric>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/pt.h"
#include "pt_host.h"
#include "pt_internal.h"
#include "pt_kernels.h"

using namespace ptg;

namespace {

// Schedule of one size: runs per CTA and, per run, either slot_parallel slots
// of L^2 threads (cell-major, team 0) or slot_parallel teams of `team` lanes
// (slot-major, at the size's largest temperature count).  block 0: the CTA
// size is the bundle's thread count rounded up to a warp.
struct ShapeSched {
    int sp = 0, ipc = 0, team = 0, block = 0;
};

struct SizeGroup {
    int L = 0, ntmax = 0, prio = 0;
    int64_t work = 0;                 // attempts per sweep
    ShapeSched s;
    std::vector<Bundle> bundles;
    Bundle* d_bundles = nullptr;
    int block = 0, smem = 0, grid = 0;
    cudaStream_t st = nullptr;        // capture branch
    cudaEvent_t ev = nullptr;
    cudaGraphNode_t knode = nullptr;
};

}  // namespace

struct pt_batch {
    int n_inst = 0, R = 0;
    uint32_t seed = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<int> L, NT, N;
    std::vector<uint32_t> uid;
    std::vector<std::vector<int8_t>> J;
    std::vector<Tables> tb;
    int kt = KT_DEFAULT;            // Metropolis table rows per slot, shared by every instance
    // device storage (one allocation per kind)
    int8_t* spins = nullptr;
    int32_t* E = nullptr;
    uint8_t* perm = nullptr;
    int32_t *best = nullptr, *first = nullptr;
    unsigned long long *macc = nullptr, *xacc = nullptr;
    uint32_t* jw = nullptr;
    uint32_t* thr = nullptr;
    int32_t* xoff = nullptr;
    uint32_t* xthr = nullptr;
    float* xhint = nullptr;
    int16_t* nbr = nullptr;
    InstDesc* d_desc = nullptr;
    int2* d_items = nullptr;
    int* d_queue = nullptr;            // one work counter per group
    int32_t* d_tts = nullptr;
    std::vector<InstDesc> desc;
    std::vector<size_t> rep_off;      // first replica of each instance
    std::vector<SizeGroup> groups;    // largest work first
    uint64_t sweep = 0;
    uint64_t launches = 0;
    // graph of {counter reset, one persistent sweep kernel per group}
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev_fork = nullptr;
    int g_nsweeps = -1, g_xevery = -1;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double last_ms = 0.0;
    std::string err = "no error";
};

namespace {

int bfail(pt_batch* b, int code, const std::string& msg)
{
    if (b) b->err = msg;
    else set_global_error(msg.c_str());
    return code;
}

int bcuda(pt_batch* b, cudaError_t e, const char* what)
{
    return bfail(b, e == cudaErrorMemoryAllocation ? PT_ERR_OOM : PT_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

#define BK(call, what)                                      \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return bcuda(b, e_, what);   \
    } while (0)

int max_temps_of(const pt_batch* b, int L)
{
    int nt = 1;
    for (int i = 0; i < b->n_inst; ++i)
        if (b->L[i] == L) nt = std::max(nt, b->NT[i]);
    return nt;
}

int group_of(const pt_batch* b, int L)
{
    for (size_t k = 0; k < b->groups.size(); ++k)
        if (b->groups[k].L == L) return (int)k;
    return -1;
}

template <class T>
cudaError_t balloc(T** p, size_t n)
{
    return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (n ? n : 1));
}

void default_shape_sched(int L, int NT, int R, bool slot_major, ShapeSched& s, int kt)
{
    const int L2 = L * L;
    s.block = 0;
    if (slot_major) {
        // teams of about L^2/16 lanes (2..32), one buffer each, widened until a
        // run has at least a warp; up to about 384 threads per CTA
        int team = 2;
        while (team < 32 && team * 16 < L2) team *= 2;
        int sp = std::max(1, NT);
        while (sp * team < 32 && team < 32) team *= 2;
        while (sp * team > 384 && sp > 1) sp = (sp + 1) / 2;
        int ipc = std::max(1, std::min(384 / (sp * team), R));
        while (ipc > 1 && bundle_smem_bytes(L, NT, ipc, team, false, kt) > 110 * 1024) --ipc;
        s.team = team;
        s.sp = sp;
        s.ipc = ipc;
        return;
    }
    // cell-major: about 256..512 threads per CTA, >= 32 per run
    int sp = std::max(1, std::min(NT, 512 / L2));
    while (sp * L2 < 32) ++sp;
    int ipc = std::max(1, std::min(512 / (sp * L2), R));
    while (ipc > 1 && bundle_smem_bytes(L, NT, ipc, 0, false, kt) > 110 * 1024) --ipc;
    s.team = 0;
    s.sp = sp;
    s.ipc = ipc;
}

// Bundle shape of one instance of group g: slot-major groups scale the team
// count to the instance's temperature count (the buffers per team of the
// group's largest count) and take more runs per CTA where that frees
// threads, within the group's shared memory at its largest count.
void instance_shape(const pt_batch* b, const SizeGroup& g, int NT, int* sp, int* ipc)
{
    const ShapeSched& s = g.s;
    if (s.team == 0) {
        *sp = s.sp;
        *ipc = std::min(s.ipc, b->R);
        return;
    }
    const int per = (g.ntmax + s.sp - 1) / s.sp;
    const int spi = std::max((NT + per - 1) / per, (32 + s.team - 1) / s.team);
    const int threads = s.sp * s.team * s.ipc;
    const int64_t smem_cap = bundle_smem_bytes(g.L, g.ntmax, s.ipc, s.team, false, b->kt);
    int ipci = std::min(s.ipc, b->R);
    while (ipci < b->R && spi * s.team * (ipci + 1) <= threads &&
           bundle_smem_bytes(g.L, NT, ipci + 1, s.team, false, b->kt) <= smem_cap)
        ++ipci;
    *sp = spi;
    *ipc = ipci;
}

// Builds group k's bundle list from its schedule and uploads it; on any
// error the group keeps its previous list, grid and CTA size.
int build_group(pt_batch* b, int k)
{
    SizeGroup& g = b->groups[k];
    const ShapeSched& s = g.s;
    const bool sm = s.team > 0;
    if (s.sp < 1 || s.ipc < 1 || (sm && (s.team > 32 || (s.team & (s.team - 1)) != 0)))
        return bfail(b, PT_ERR_ARG, "bad schedule values");
    if ((sm ? s.sp * s.team : s.sp * g.L * g.L) < 32)
        return bfail(b, PT_ERR_ARG, "schedule of L=" + std::to_string(g.L) + " does not fit (threads per run >= 32)");
    std::vector<Bundle> bundles;
    int threads = 0;
    int64_t smem = 0;
    for (int i = 0; i < b->n_inst; ++i) {
        if (b->L[i] != g.L) continue;
        int spi = 0, ipci = 0;
        instance_shape(b, g, b->NT[i], &spi, &ipci);
        const int tpr = sm ? spi * s.team : spi * g.L * g.L;
        if (tpr < 32)
            return bfail(b, PT_ERR_ARG, "schedule of L=" + std::to_string(g.L) + " does not fit (threads per run >= 32)");
        for (int r = 0; r < b->R; r += ipci) {
            Bundle bd;
            bd.inst = i; bd.run0 = r; bd.nitems = std::min(ipci, b->R - r); bd.sp = spi; bd.team = s.team;
            bundles.push_back(bd);
        }
        threads = std::max(threads, tpr * ipci);
        smem = std::max<int64_t>(smem, bundle_smem_bytes(g.L, b->NT[i], ipci, s.team, false, b->kt));
    }
    int block = (threads + 31) / 32 * 32;
    if (s.block > 0) {
        if (s.block < block || s.block % 32 != 0)
            return bfail(b, PT_ERR_ARG, "schedule of L=" + std::to_string(g.L) + " does not fit the block");
        block = s.block;
    }
    if (block > (sm ? MAX_THREADS_SM : MAX_THREADS))
        return bfail(b, PT_ERR_ARG, "schedule of L=" + std::to_string(g.L) + " does not fit: " +
                                        std::to_string(block) + " threads per CTA (limit " +
                                        std::to_string(sm ? MAX_THREADS_SM : MAX_THREADS) + ")");
    // longest bundles first (work per sweep = runs x slots x spins)
    std::stable_sort(bundles.begin(), bundles.end(), [&](const Bundle& x, const Bundle& y) {
        const int64_t cx = (int64_t)x.nitems * b->NT[x.inst] * b->N[x.inst];
        const int64_t cy = (int64_t)y.nitems * b->NT[y.inst] * b->N[y.inst];
        return cx > cy;
    });
    int cap = 0;
    BK(sweep_smem_capacity(&cap), "shared memory capacity");
    if (smem > cap) return bfail(b, PT_ERR_ARG, "a bundle needs more shared memory than a CTA can have");
    BK(set_sweep_smem_limit(cap), "cudaFuncSetAttribute");
    int dev = 0, sms = 0, per_sm = 0;
    BK(cudaGetDevice(&dev), "cudaGetDevice");
    BK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device attribute");
    BK(sweep_occupancy(block, (int)smem, &per_sm, sm), "occupancy");
    if (per_sm < 1) return bfail(b, PT_ERR_ARG, "schedule of L=" + std::to_string(g.L) + " fits no CTA on an SM");
    Bundle* d = nullptr;
    BK(balloc(&d, bundles.size()), "cudaMalloc bundles");
    cudaError_t e = cudaMemcpyAsync(d, bundles.data(), sizeof(Bundle) * bundles.size(), cudaMemcpyHostToDevice,
                                    b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) { cudaFree(d); return bcuda(b, e, "upload bundles"); }
    cudaFree(g.d_bundles);
    g.d_bundles = d;
    g.bundles.swap(bundles);
    g.block = block;
    g.smem = (int)smem;
    g.grid = std::max(1, std::min<int>((int)g.bundles.size(), sms * per_sm));
    // the captured graph holds the old bundle lists
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    b->g_nsweeps = b->g_xevery = -1;
    return PT_OK;
}

// Sets group k's schedule and rebuilds it, keeping the old one on failure.
int set_group(pt_batch* b, int k, const ShapeSched& s)
{
    const ShapeSched old = b->groups[k].s;
    b->groups[k].s = s;
    const int rc = build_group(b, k);
    if (rc) b->groups[k].s = old;
    return rc;
}

int run_graph(pt_batch* b, int nsweeps, int xevery)
{
    const int ng = (int)b->groups.size();
    if (!b->exec || b->g_nsweeps != nsweeps || b->g_xevery != xevery) {
        if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
        if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
        cudaStream_t cs;
        BK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream");
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->d_queue, 0, sizeof(int) * ng, cs);
        if (e == cudaSuccess) e = cudaEventRecord(b->ev_fork, cs);
        for (int k = 0; k < ng && e == cudaSuccess; ++k) {
            SizeGroup& g = b->groups[k];
            e = cudaStreamWaitEvent(g.st, b->ev_fork, 0);
            if (e == cudaSuccess)
                e = launch_sweeps(b->d_desc, g.d_bundles, (int)g.bundles.size(), g.grid, g.block, g.smem,
                                  (uint32_t)b->sweep, nsweeps, xevery, 0, b->d_queue + k, g.st, g.s.team > 0, false,
                                  g.L);
            if (e == cudaSuccess) e = cudaEventRecord(g.ev, g.st);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, g.ev, 0);
        }
        cudaGraph_t gr = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cs, &gr);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) { if (gr) cudaGraphDestroy(gr); return bcuda(b, e, "graph capture"); }
        if (e2 != cudaSuccess) return bcuda(b, e2, "end capture");
        b->graph = gr;
        size_t n = 0;
        BK(cudaGraphGetNodes(gr, nullptr, &n), "graph nodes");
        std::vector<cudaGraphNode_t> nodes(n);
        BK(cudaGraphGetNodes(gr, nodes.data(), &n), "graph nodes");
        for (auto& g : b->groups) g.knode = nullptr;
        for (auto nd : nodes) {                  // a kernel node is known by its work counter
            cudaGraphNodeType t;
            BK(cudaGraphNodeGetType(nd, &t), "node type");
            if (t != cudaGraphNodeTypeKernel) continue;
            cudaKernelNodeParams kp;
            BK(cudaGraphKernelNodeGetParams(nd, &kp), "kernel node params");
            const int* q = *reinterpret_cast<int* const*>(kp.kernelParams[7]);
            const long k = (long)(q - b->d_queue);
            if (k >= 0 && k < ng) b->groups[k].knode = nd;
        }
        for (auto& g : b->groups) {
            if (!g.knode) return bfail(b, PT_ERR_CUDA, "captured graph lacks a group's kernel node");
            cudaKernelNodeAttrValue v;
            std::memset(&v, 0, sizeof(v));
            v.priority = g.prio;
            BK(cudaGraphKernelNodeSetAttribute(g.knode, cudaKernelNodeAttributePriority, &v), "node priority");
        }
        BK(cudaGraphInstantiate(&b->exec, gr, 0), "graph instantiate");
        b->g_nsweeps = nsweeps;
        b->g_xevery = xevery;
    }
    // patch the sweep counter (argument 3 of pt_sweep_kernel) and replay
    uint32_t sweep0 = (uint32_t)b->sweep;
    for (auto& g : b->groups) {
        cudaKernelNodeParams kp;
        BK(cudaGraphKernelNodeGetParams(g.knode, &kp), "kernel node params");
        void* args[8];
        for (int i = 0; i < 8; ++i) args[i] = kp.kernelParams[i];
        args[3] = &sweep0;
        kp.kernelParams = args;
        BK(cudaGraphExecKernelNodeSetParams(b->exec, g.knode, &kp), "patch kernel node");
    }
    BK(cudaGraphLaunch(b->exec, b->stream), "graph launch");
    BK(debug_check(b->stream, "batched sweep graph"), "debug check");
    b->launches += (uint64_t)b->groups.size();
    return PT_OK;
}

}  // namespace

extern "C" {

const char* pt_batch_last_error(const pt_batch* b)
{
    return b ? b->err.c_str() : pt_last_error(nullptr);
}

int pt_batch_create(pt_batch** out, int32_t n_inst, const pt_instance_desc* d, int32_t n_runs,
                    uint32_t seed, void* stream)
{
    pt_batch* b = nullptr;
    if (!out || !d) return bfail(nullptr, PT_ERR_ARG, "NULL argument");
    *out = nullptr;
    if (n_inst < 1 || n_inst > 65536) return bfail(nullptr, PT_ERR_ARG, "n_inst must be in [1, 65536]");
    if (n_runs < 1 || n_runs > 1024) return bfail(nullptr, PT_ERR_ARG, "n_runs must be in [1, 1024]");
    b = new (std::nothrow) pt_batch();
    if (!b) return bfail(nullptr, PT_ERR_OOM, "host allocation failed");
    auto bail = [&](int code) { std::string m = b->err; pt_batch_destroy(b); return bfail(nullptr, code, m); };
    b->n_inst = n_inst; b->R = n_runs; b->seed = seed;
    for (int i = 0; i < n_inst; ++i) {
        const pt_instance_desc& x = d[i];
        if (x.chimera_L < 1 || x.chimera_L > MAX_L || !x.J || !x.betas || x.n_temps < 1 || x.n_temps > MAX_TEMPS) {
            b->err = "instance " + std::to_string(i) + ": bad L, n_temps or NULL array";
            return bail(PT_ERR_ARG);
        }
        const int E = n_edges_of(x.chimera_L);
        for (int e = 0; e < E; ++e)
            if (x.J[e] < -J_ABS_MAX) { b->err = "instance " + std::to_string(i) + ": coupler outside [-127, 127]"; return bail(PT_ERR_ARG); }
        const int km = coupler_kmax(x.chimera_L, x.J);
        if (km > KT_MAX - 1) { b->err = "instance " + std::to_string(i) + ": a spin's sum of |J| exceeds 127"; return bail(PT_ERR_ARG); }
        b->kt = std::max(b->kt, table_rows_for(km));
        for (int t = 0; t < x.n_temps; ++t)
            if (!(x.betas[t] > 0.0) || !std::isfinite(x.betas[t]) || (t > 0 && !(x.betas[t] < x.betas[t - 1]))) {
                b->err = "instance " + std::to_string(i) + ": betas must be finite, > 0, strictly descending";
                return bail(PT_ERR_ARG);
            }
        b->L.push_back(x.chimera_L);
        b->NT.push_back(x.n_temps);
        b->N.push_back(8 * x.chimera_L * x.chimera_L);
        b->uid.push_back(x.uid);
        b->J.emplace_back(x.J, x.J + E);
    }
    // one table row count for the whole batch: the largest any instance needs
    for (int i = 0; i < n_inst; ++i) {
        const pt_instance_desc& x = d[i];
        Tables tb;
        std::string why = build_tables(x.n_temps, b->kt, x.betas, tb);
        if (!why.empty()) { b->err = "instance " + std::to_string(i) + ": " + why; return bail(PT_ERR_ARG); }
        b->tb.push_back(std::move(tb));
    }
    if (stream) b->stream = (cudaStream_t)stream;
    else {
        cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { bcuda(b, e, "cudaStreamCreate"); return bail(PT_ERR_CUDA); }
        b->own_stream = true;
    }
#define BKC(call, what)                                                          \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) { int c_ = bcuda(b, e_, what); return bail(c_); } \
    } while (0)
    size_t reps = 0, runs = (size_t)n_inst * n_runs, pairs = 0, jws = 0, thrs = 0, xts = 0, nts = 0;
    for (int i = 0; i < n_inst; ++i) {
        b->rep_off.push_back(reps);
        reps += (size_t)n_runs * b->NT[i];
        pairs += (size_t)n_runs * std::max(b->NT[i] - 1, 1);
        jws += (size_t)b->L[i] * b->L[i] * 16;
        thrs += (size_t)b->NT[i] * b->kt;
        xts += b->tb[i].xthr.size();
        nts += (size_t)b->NT[i];
    }
    size_t spin_bytes = 0;
    for (int i = 0; i < n_inst; ++i) spin_bytes += (size_t)n_runs * b->NT[i] * b->N[i];
    BKC(balloc(&b->spins, spin_bytes), "cudaMalloc spins");
    BKC(balloc(&b->E, reps), "cudaMalloc E");
    BKC(balloc(&b->perm, reps), "cudaMalloc perm");
    BKC(balloc(&b->best, runs), "cudaMalloc best");
    BKC(balloc(&b->first, runs), "cudaMalloc first");
    BKC(balloc(&b->macc, reps), "cudaMalloc macc");
    BKC(balloc(&b->xacc, pairs), "cudaMalloc xacc");
    BKC(balloc(&b->jw, jws), "cudaMalloc jw");
    BKC(balloc(&b->thr, thrs), "cudaMalloc thr");
    BKC(balloc(&b->xoff, nts), "cudaMalloc xoff");
    BKC(balloc(&b->xhint, nts), "cudaMalloc xhint");
    BKC(balloc(&b->xthr, xts), "cudaMalloc xthr");
    BKC(balloc(&b->nbr, (size_t)(MAX_L + 1) * MAX_L * MAX_L * 4), "cudaMalloc nbr");
    BKC(balloc(&b->d_desc, (size_t)n_inst), "cudaMalloc desc");
    BKC(balloc(&b->d_items, runs), "cudaMalloc items");
    std::map<int, int> sizes;                                    // L -> instances
    for (int i = 0; i < n_inst; ++i) sizes[b->L[i]] += 1;
    BKC(balloc(&b->d_queue, sizes.size()), "cudaMalloc queues");
    BKC(balloc(&b->d_tts, (size_t)n_inst * 3), "cudaMalloc tts");
    BKC(cudaEventCreate(&b->e0), "event");
    BKC(cudaEventCreate(&b->e1), "event");
    // per-L neighbour tables
    std::vector<int16_t> nb((size_t)MAX_L * MAX_L * 4);
    for (int L = 1; L <= MAX_L; ++L) {
        build_neighbours(L, nb.data());
        BKC(cudaMemcpy(b->nbr + (size_t)L * MAX_L * MAX_L * 4, nb.data(), 2 * (size_t)L * L * 4,
                       cudaMemcpyHostToDevice), "upload nbr");
    }
    size_t o_sp = 0, o_jw = 0, o_thr = 0, o_xt = 0, o_nt = 0, o_pair = 0;
    std::vector<int2> items;
    for (int i = 0; i < n_inst; ++i) {
        const int L = b->L[i], NT = b->NT[i];
        InstDesc dd;
        dd.L = L; dd.NT = NT; dd.R = n_runs; dd.n_xpairs = NT - 1;
        dd.seed = seed; dd.uid = b->uid[i];
        dd.kt = b->kt;
        std::vector<uint32_t> jw((size_t)L * L * 16);
        pack_couplers(L, b->J[i].data(), jw.data());
        BKC(cudaMemcpy(b->jw + o_jw, jw.data(), 4 * jw.size(), cudaMemcpyHostToDevice), "upload jw");
        BKC(cudaMemcpy(b->thr + o_thr, b->tb[i].thr.data(), 4 * b->tb[i].thr.size(), cudaMemcpyHostToDevice), "upload thr");
        std::vector<int32_t> xo(b->tb[i].xoff.begin(), b->tb[i].xoff.end());
        BKC(cudaMemcpy(b->xoff + o_nt, xo.data(), 4 * xo.size(), cudaMemcpyHostToDevice), "upload xoff");
        BKC(cudaMemcpy(b->xhint + o_nt, b->tb[i].xhint.data(), 4 * std::min<size_t>(b->tb[i].xhint.size(), NT),
                       cudaMemcpyHostToDevice), "upload xhint");
        if (!b->tb[i].xthr.empty())
            BKC(cudaMemcpy(b->xthr + o_xt, b->tb[i].xthr.data(), 4 * b->tb[i].xthr.size(), cudaMemcpyHostToDevice), "upload xthr");
        dd.jw = b->jw + o_jw;
        dd.nbr = b->nbr + (size_t)L * MAX_L * MAX_L * 4;
        dd.thr = b->thr + o_thr;
        dd.xoff = b->xoff + o_nt;
        dd.xthr = b->xthr + o_xt;
        dd.xhint = b->xhint + o_nt;
        dd.spins = b->spins + o_sp;
        dd.E = b->E + b->rep_off[i];
        dd.perm = b->perm + b->rep_off[i];
        dd.best = b->best + (size_t)i * n_runs;
        dd.first = b->first + (size_t)i * n_runs;
        dd.macc = b->macc + b->rep_off[i];
        dd.xacc = b->xacc + o_pair;
        b->desc.push_back(dd);
        o_sp += (size_t)n_runs * NT * b->N[i];
        o_jw += jw.size();
        o_thr += b->tb[i].thr.size();
        o_xt += b->tb[i].xthr.size();
        o_nt += (size_t)NT;
        o_pair += (size_t)n_runs * std::max(NT - 1, 1);
        for (int r = 0; r < n_runs; ++r) items.push_back(make_int2(i, r));
    }
    // one group per size, largest work first (that order is also the
    // branches' stream priority order)
    for (auto& kv : sizes) {
        SizeGroup g;
        g.L = kv.first;
        g.ntmax = max_temps_of(b, g.L);
        for (int i = 0; i < n_inst; ++i)
            if (b->L[i] == g.L) g.work += (int64_t)n_runs * b->NT[i] * b->N[i];
        default_shape_sched(g.L, g.ntmax, n_runs, false, g.s, b->kt);
        b->groups.push_back(g);
    }
    std::stable_sort(b->groups.begin(), b->groups.end(),
                     [](const SizeGroup& x, const SizeGroup& y) { return x.work > y.work; });
    int prio_least = 0, prio_greatest = 0;
    BKC(cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest), "stream priorities");
    for (size_t k = 0; k < b->groups.size(); ++k) {
        SizeGroup& g = b->groups[k];
        g.prio = std::min(prio_least, prio_greatest + (int)k);
        BKC(cudaStreamCreateWithPriority(&g.st, cudaStreamNonBlocking, g.prio), "group stream");
        BKC(cudaEventCreateWithFlags(&g.ev, cudaEventDisableTiming), "group event");
    }
    BKC(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming), "fork event");
    BKC(cudaMemcpy(b->d_desc, b->desc.data(), sizeof(InstDesc) * b->desc.size(), cudaMemcpyHostToDevice), "upload desc");
    BKC(cudaMemcpy(b->d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice), "upload items");
    for (size_t k = 0; k < b->groups.size(); ++k) {
        int rc = build_group(b, (int)k);
        if (rc) return bail(rc);
    }
    int rc = PT_OK;
    rc = pt_batch_reset(b);
    if (rc) return bail(rc);
#undef BKC
    *out = b;
    return PT_OK;
}

void pt_batch_destroy(pt_batch* b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto& g : b->groups) {
        cudaFree(g.d_bundles);
        if (g.st) cudaStreamDestroy(g.st);
        if (g.ev) cudaEventDestroy(g.ev);
    }
    cudaFree(b->spins); cudaFree(b->E); cudaFree(b->perm); cudaFree(b->best); cudaFree(b->first);
    cudaFree(b->macc); cudaFree(b->xacc); cudaFree(b->jw); cudaFree(b->thr); cudaFree(b->xoff);
    cudaFree(b->xthr); cudaFree(b->xhint); cudaFree(b->nbr); cudaFree(b->d_desc); cudaFree(b->d_items);
    cudaFree(b->d_queue); cudaFree(b->d_tts);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->e0) cudaEventDestroy(b->e0);
    if (b->e1) cudaEventDestroy(b->e1);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

int pt_batch_reset(pt_batch* b)
{
    if (!b) return PT_ERR_ARG;
    const int nitems = b->n_inst * b->R;
    BK(launch_init(b->d_desc, b->d_items, nitems, true, b->stream), "init kernel");
    BK(launch_energy(b->d_desc, b->d_items, nitems, 0, b->stream), "energy kernel");
    b->launches += 2;
    b->sweep = 0;
    BK(cudaStreamSynchronize(b->stream), "sync reset");
    return PT_OK;
}

int pt_batch_run(pt_batch* b, int32_t n_sweeps, int32_t exchange_every)
{
    if (!b) return PT_ERR_ARG;
    if (n_sweeps < 0 || n_sweeps > (1 << 24) || exchange_every < 0)
        return bfail(b, PT_ERR_ARG, "n_sweeps must be in [0, 2^24], exchange_every >= 0");
    if (b->sweep + (uint64_t)n_sweeps > 0x7FFFFFFFull) return bfail(b, PT_ERR_STATE, "sweep counter would exceed 2^31-1");
    if (n_sweeps == 0) return PT_OK;
    BK(cudaEventRecord(b->e0, b->stream), "event");
    int rc = run_graph(b, n_sweeps, exchange_every);
    if (rc) return rc;
    BK(cudaEventRecord(b->e1, b->stream), "event");
    BK(cudaStreamSynchronize(b->stream), "sync run");
    float ms = 0.f;
    BK(cudaEventElapsedTime(&ms, b->e0, b->e1), "event time");
    b->last_ms = ms;
    b->sweep += (uint64_t)n_sweeps;
    return PT_OK;
}

int pt_batch_tts(pt_batch* b, int32_t horizon, int32_t* tts, int32_t* n_hit, int32_t* target)
{
    if (!b || !tts) return bfail(b, PT_ERR_ARG, "NULL argument");
    BK(launch_tts(b->d_desc, b->n_inst, PT_TARGET_BEST, horizon, b->d_tts, b->stream), "tts kernel");
    b->launches += 1;
    std::vector<int32_t> out((size_t)b->n_inst * 3);
    BK(cudaMemcpyAsync(out.data(), b->d_tts, 4 * out.size(), cudaMemcpyDeviceToHost, b->stream), "download tts");
    BK(cudaStreamSynchronize(b->stream), "sync tts");
    for (int i = 0; i < b->n_inst; ++i) {
        tts[i] = out[(size_t)i * 3];
        if (n_hit) n_hit[i] = out[(size_t)i * 3 + 1];
        if (target) target[i] = out[(size_t)i * 3 + 2];
    }
    return PT_OK;
}

int pt_batch_get_state(pt_batch* b, int32_t inst, int8_t* spins, int32_t* E, int32_t* best, int32_t* first,
                       uint64_t* macc, uint64_t* xacc)
{
    if (!b || inst < 0 || inst >= b->n_inst) return bfail(b, PT_ERR_ARG, "instance index out of range");
    const InstDesc& d = b->desc[inst];
    const size_t reps = (size_t)b->R * d.NT, N = 8 * (size_t)d.L * d.L;
    std::vector<uint8_t> pm(reps);
    std::vector<int8_t> sp;
    BK(cudaMemcpyAsync(pm.data(), d.perm, reps, cudaMemcpyDeviceToHost, b->stream), "download perm");
    if (spins) {
        sp.resize(reps * N);
        BK(cudaMemcpyAsync(sp.data(), d.spins, reps * N, cudaMemcpyDeviceToHost, b->stream), "download spins");
    }
    if (E) BK(cudaMemcpyAsync(E, d.E, 4 * reps, cudaMemcpyDeviceToHost, b->stream), "download E");
    if (best) BK(cudaMemcpyAsync(best, d.best, 4 * (size_t)b->R, cudaMemcpyDeviceToHost, b->stream), "download best");
    if (first) BK(cudaMemcpyAsync(first, d.first, 4 * (size_t)b->R, cudaMemcpyDeviceToHost, b->stream), "download first");
    if (macc) BK(cudaMemcpyAsync(macc, d.macc, 8 * reps, cudaMemcpyDeviceToHost, b->stream), "download macc");
    if (xacc && d.NT > 1)
        BK(cudaMemcpyAsync(xacc, d.xacc, 8 * (size_t)b->R * (d.NT - 1), cudaMemcpyDeviceToHost, b->stream), "download xacc");
    BK(cudaStreamSynchronize(b->stream), "sync get_state");
    if (spins)
        for (int r = 0; r < b->R; ++r)
            for (int t = 0; t < d.NT; ++t)
                std::memcpy(spins + ((size_t)r * d.NT + t) * N,
                            sp.data() + ((size_t)r * d.NT + pm[(size_t)r * d.NT + t]) * N, N);
    return PT_OK;
}

int pt_batch_set_schedule(pt_batch* b, int32_t block, int32_t chimera_L, int32_t slot_parallel, int32_t runs_per_cta)
{
    if (!b) return PT_ERR_ARG;
    if (block < 0 || block % 32 != 0 || block > MAX_THREADS)
        return bfail(b, PT_ERR_ARG, "block must be 0 or a multiple of 32, <= 1024");
    if (chimera_L <= 0) {                  // CTA size of every size (validated group by group)
        std::vector<ShapeSched> old;
        for (auto& g : b->groups) old.push_back(g.s);
        for (size_t k = 0; k < b->groups.size(); ++k) {
            ShapeSched s = b->groups[k].s;
            s.block = block;
            const int rc = set_group(b, (int)k, s);
            if (rc) {
                for (size_t m = 0; m < k; ++m) set_group(b, (int)m, old[m]);
                return rc;
            }
        }
    } else {
        const int k = group_of(b, chimera_L);
        if (k < 0) return bfail(b, PT_ERR_ARG, "no instance of that size");
        if (slot_parallel < 1 || runs_per_cta < 1) return bfail(b, PT_ERR_ARG, "slot_parallel, runs_per_cta must be >= 1");
        ShapeSched s = b->groups[k].s;
        s.sp = slot_parallel;
        s.ipc = std::min<int>(runs_per_cta, b->R);
        s.block = block;
        const int rc = set_group(b, k, s);
        if (rc) return rc;
    }
    BK(cudaStreamSynchronize(b->stream), "sync schedule");
    return PT_OK;
}

int pt_batch_set_mapping(pt_batch* b, int32_t chimera_L, int32_t team, int32_t slot_parallel, int32_t runs_per_cta)
{
    if (!b || team < 0) return bfail(b, PT_ERR_ARG, "team must be >= 0");
    if (team > 0 && (team > 32 || (team & (team - 1)) != 0))
        return bfail(b, PT_ERR_ARG, "team must be a power of two <= 32");
    if (chimera_L <= 0) {                  // every size: the mapping's default schedule
        std::vector<ShapeSched> old;
        for (auto& g : b->groups) old.push_back(g.s);
        for (size_t k = 0; k < b->groups.size(); ++k) {
            SizeGroup& g = b->groups[k];
            ShapeSched s;
            default_shape_sched(g.L, g.ntmax, b->R, team > 0, s, b->kt);
            const int rc = set_group(b, (int)k, s);
            if (rc) {
                for (size_t m = 0; m < k; ++m) set_group(b, (int)m, old[m]);
                return rc;
            }
        }
    } else {
        const int k = group_of(b, chimera_L);
        if (k < 0) return bfail(b, PT_ERR_ARG, "no instance of that size");
        SizeGroup& g = b->groups[k];
        ShapeSched s = g.s;
        if ((s.team > 0) != (team > 0)) default_shape_sched(g.L, g.ntmax, b->R, team > 0, s, b->kt);
        if (team > 0) s.team = team;
        if (slot_parallel > 0) s.sp = slot_parallel;
        if (runs_per_cta > 0) s.ipc = std::min<int>(runs_per_cta, b->R);
        s.block = 0;
        const int rc = set_group(b, k, s);
        if (rc) return rc;
    }
    BK(cudaStreamSynchronize(b->stream), "sync mapping");
    return PT_OK;
}

int pt_batch_get_schedule(const pt_batch* b, int32_t chimera_L, int32_t* block, int32_t* slot_parallel,
                          int32_t* runs_per_cta)
{
    if (!b) return PT_ERR_ARG;
    const int k = group_of(b, chimera_L);
    if (k < 0) return PT_ERR_ARG;
    const SizeGroup& g = b->groups[k];
    if (block) *block = g.block;
    if (slot_parallel) *slot_parallel = g.s.sp;
    if (runs_per_cta) *runs_per_cta = g.s.ipc;
    return PT_OK;
}

int pt_batch_get_mapping(const pt_batch* b, int32_t chimera_L, int32_t* team)
{
    if (!b) return PT_ERR_ARG;
    const int k = group_of(b, chimera_L);
    if (k < 0) return PT_ERR_ARG;
    if (team) *team = b->groups[k].s.team;
    return PT_OK;
}

// Times candidate schedules and keeps the fastest, size by size: every
// cell-major (slot_parallel, runs_per_cta) and slot-major (team,
// slot_parallel, runs_per_cta) that fits runs all instances of that size
// alone for `trial_sweeps` sweeps (the faster of two launches), with the CTA
// size the bundle needs.  The state is reset afterwards.
int pt_batch_autotune(pt_batch* b, int32_t trial_sweeps, int32_t* block_out)
{
    if (!b || trial_sweeps < 1) return bfail(b, PT_ERR_ARG, "need trial_sweeps >= 1");
    int cap = 0;
    BK(sweep_smem_capacity(&cap), "shared memory capacity");
    for (size_t k = 0; k < b->groups.size(); ++k) {
        SizeGroup& g = b->groups[k];
        const int L2 = g.L * g.L, NT = g.ntmax;
        std::vector<ShapeSched> cands;
        for (int sp : {1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64}) {
            const int tpr = sp * L2;
            if (sp > NT || tpr > MAX_THREADS) break;
            if (tpr < 32) continue;
            for (int ipc : {1, 2, 4, 8, 16}) {
                if (tpr * ipc > MAX_THREADS || ipc > b->R || bundle_smem_bytes(g.L, NT, ipc, 0, false, b->kt) > cap) break;
                ShapeSched s; s.sp = sp; s.ipc = ipc; s.team = 0;
                cands.push_back(s);
            }
        }
        for (int team : {2, 4, 8, 16, 32}) {
            if (team > 2 * L2) break;
            int prev = 0;
            for (int nt : {NT, (NT + 1) / 2, (NT + 3) / 4, (NT + 7) / 8}) {
                if (nt == prev || nt * team < 32 || nt * team > MAX_THREADS_SM) continue;
                prev = nt;
                for (int ipc : {1, 2, 4, 8}) {
                    if (nt * team * ipc > MAX_THREADS_SM || ipc > b->R ||
                        bundle_smem_bytes(g.L, NT, ipc, team, false, b->kt) > cap)
                        break;
                    ShapeSched s; s.sp = nt; s.ipc = ipc; s.team = team;
                    cands.push_back(s);
                }
            }
        }
        const ShapeSched old = g.s;
        double best_rate = 0.0;
        ShapeSched best = old;
        for (const ShapeSched& c : cands) {
            if (set_group(b, (int)k, c) != PT_OK) continue;
            const double att = (double)g.work * trial_sweeps;
            float ms = 1e30f;
            for (int rep = 0; rep < 2; ++rep) {      // the faster of two launches
                cudaError_t e = cudaEventRecord(b->e0, b->stream);
                if (e == cudaSuccess) e = cudaMemsetAsync(b->d_queue + k, 0, sizeof(int), b->stream);
                if (e == cudaSuccess)
                    e = launch_sweeps(b->d_desc, g.d_bundles, (int)g.bundles.size(), g.grid, g.block, g.smem, 0u,
                                      trial_sweeps, 1, 0, b->d_queue + k, b->stream, g.s.team > 0, false, g.L);
                if (e == cudaSuccess) e = cudaEventRecord(b->e1, b->stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(b->e1);
                float t = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&t, b->e0, b->e1);
                if (e != cudaSuccess) {
                    const int code = bcuda(b, e, "trial launch");
                    set_group(b, (int)k, old);
                    return code;
                }
                ms = std::min(ms, t);
            }
            const double rate = att / (ms * 1e-3);
            if (rate > best_rate) { best_rate = rate; best = c; }
        }
        const int rc = set_group(b, (int)k, best);
        if (rc) { set_group(b, (int)k, old); return rc; }
    }
    const int rc = pt_batch_reset(b);
    if (rc) return rc;
    if (block_out) *block_out = b->groups.empty() ? 0 : b->groups[0].block;
    return PT_OK;
}

int pt_batch_info(const pt_batch* b, double* last_run_ms, int32_t* grid, int32_t* block, int32_t* n_bundles,
                  uint64_t* launches)
{
    if (!b) return PT_ERR_ARG;
    int gsum = 0, bmax = 0, nb = 0;
    for (const auto& g : b->groups) {
        gsum += g.grid;
        bmax = std::max(bmax, g.block);
        nb += (int)g.bundles.size();
    }
    if (last_run_ms) *last_run_ms = b->last_ms;
    if (grid) *grid = gsum;
    if (block) *block = bmax;
    if (n_bundles) *n_bundles = nb;
    if (launches) *launches = b->launches;
    return PT_OK;
}

}  // extern "C"
