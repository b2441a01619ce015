// pt_batch.cu -- batched PT of many instances of uneven size and temperature
// count in one persistent, graph-captured launch (C ABI: pt_batch_* in pt.h).
//
// Every (instance, run) pair is an independent PT run (Sec. II); the host packs
// them into CTA bundles (a few runs of one instance), orders the bundles by
// cost (longest first), and one persistent kernel grid pulls bundles from an
// atomic counter until none is left.  The queue reset and the launch are
// captured once in a CUDA graph; each pt_batch_run replays it with the sweep
// counter patched into the kernel node.  Schedules per Chimera size (threads
// per run, runs per CTA) come from pt_batch_autotune and never change results.
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

// Per Chimera size: runs per CTA and, per run, either slot_parallel slots of
// L^2 threads (cell-major, team 0) or slot_parallel teams of `team` lanes
// (slot-major).  All sizes of a batch share one mapping: one launch runs one
// kernel instantiation.
struct ShapeSched {
    int sp = 0, ipc = 0, team = 0;
};

int sched_threads(int L, const ShapeSched& s)
{
    return s.team > 0 ? s.sp * s.team : s.sp * L * L;
}

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
    Bundle* d_bundles = nullptr;
    int* d_queue = nullptr;
    int32_t* d_tts = nullptr;
    std::vector<InstDesc> desc;
    std::vector<size_t> rep_off;      // first replica of each instance
    std::map<int, ShapeSched> sched;  // per L
    int block = 512;
    bool slot_major = false;
    std::vector<Bundle> bundles;
    int smem = 0, grid = 0;
    uint64_t sweep = 0;
    uint64_t launches = 0;
    // graph of {queue reset, persistent sweep kernel}
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t knode = nullptr;
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

template <class T>
cudaError_t balloc(T** p, size_t n)
{
    return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (n ? n : 1));
}

void default_shape_sched(int L, int NT, int R, int block, bool slot_major, ShapeSched& s)
{
    const int L2 = L * L;
    if (slot_major) {
        // one team of 4 lanes per slot (2 for the single-cell lattice), widened
        // until a run has at least a warp
        int team = L2 >= 4 ? 4 : 2, sp = std::max(1, NT);
        while (sp * team < 32 && team < 32) team *= 2;
        while (sp * team > block && sp > 1) sp = (sp + 1) / 2;
        int ipc = std::max(1, std::min(block / (sp * team), R));
        while (ipc > 1 && bundle_smem_bytes(L, NT, ipc, team) > 110 * 1024) --ipc;
        s.team = team;
        s.sp = sp;
        s.ipc = ipc;
        return;
    }
    // about block/2 .. block threads per CTA, >= 32 threads per run
    int sp = std::max(1, std::min(NT, block / L2));
    while (sp * L2 < 32) ++sp;
    if (sp * L2 > block) sp = std::max(1, block / L2);
    int ipc = std::max(1, block / (sp * L2));
    ipc = std::min(ipc, R);
    while (ipc > 1 && bundle_smem_bytes(L, NT, ipc) > 110 * 1024) --ipc;
    s.team = 0;
    s.sp = sp;
    s.ipc = ipc;
}

// Builds the bundle list of the current schedules (optionally only the sizes
// in only_L) and uploads it; on any error the previous list, grid and graph
// stay as they were.
int build_bundles(pt_batch* b, const std::vector<int>* only_L = nullptr, int max_inst_per_L = 0)
{
    std::vector<Bundle> bundles;
    std::map<int, int> taken;
    int smem = 0;
    for (int i = 0; i < b->n_inst; ++i) {
        const int L = b->L[i];
        if (only_L && std::find(only_L->begin(), only_L->end(), L) == only_L->end()) continue;
        if (max_inst_per_L > 0 && taken[L]++ >= max_inst_per_L) continue;
        const ShapeSched& s = b->sched[L];
        for (int r = 0; r < b->R; r += s.ipc) {
            Bundle bd;
            bd.inst = i; bd.run0 = r; bd.nitems = std::min(s.ipc, b->R - r); bd.sp = s.sp;
            bd.team = b->slot_major ? s.team : 0;
            bundles.push_back(bd);
        }
        if (sched_threads(L, s) * s.ipc > b->block || (b->slot_major != (s.team > 0)))
            return bfail(b, PT_ERR_ARG, "schedule of L=" + std::to_string(L) + " does not fit the block or mapping");
        smem = std::max<int>(smem, (int)bundle_smem_bytes(L, b->NT[i], s.ipc, b->slot_major ? s.team : 0));
    }
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
    BK(sweep_occupancy(b->block, smem, &per_sm, b->slot_major), "occupancy");
    Bundle* d = nullptr;
    BK(balloc(&d, bundles.size()), "cudaMalloc bundles");
    cudaError_t e = cudaMemcpyAsync(d, bundles.data(), sizeof(Bundle) * bundles.size(), cudaMemcpyHostToDevice,
                                    b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) { cudaFree(d); return bcuda(b, e, "upload bundles"); }
    cudaFree(b->d_bundles);
    b->d_bundles = d;
    b->bundles.swap(bundles);
    b->smem = smem;
    b->grid = std::max(1, std::min<int>((int)b->bundles.size(), sms * std::max(1, per_sm)));
    // the captured graph holds the old bundle list
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    b->g_nsweeps = b->g_xevery = -1;
    return PT_OK;
}

int run_graph(pt_batch* b, int nsweeps, int xevery)
{
    if (!b->exec || b->g_nsweeps != nsweeps || b->g_xevery != xevery) {
        if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
        if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
        cudaStream_t cs;
        BK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream");
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->d_queue, 0, sizeof(int), cs);
        if (e == cudaSuccess)
            e = launch_sweeps(b->d_desc, b->d_bundles, (int)b->bundles.size(), b->grid, b->block, b->smem,
                              (uint32_t)b->sweep, nsweeps, xevery, 0, b->d_queue, cs, b->slot_major);
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return bcuda(b, e, "graph capture"); }
        if (e2 != cudaSuccess) return bcuda(b, e2, "end capture");
        b->graph = g;
        size_t n = 0;
        BK(cudaGraphGetNodes(g, nullptr, &n), "graph nodes");
        std::vector<cudaGraphNode_t> nodes(n);
        BK(cudaGraphGetNodes(g, nodes.data(), &n), "graph nodes");
        b->knode = nullptr;
        for (auto nd : nodes) {
            cudaGraphNodeType t;
            BK(cudaGraphNodeGetType(nd, &t), "node type");
            if (t == cudaGraphNodeTypeKernel) b->knode = nd;
        }
        if (!b->knode) return bfail(b, PT_ERR_CUDA, "captured graph has no kernel node");
        BK(cudaGraphInstantiate(&b->exec, g, 0), "graph instantiate");
        b->g_nsweeps = nsweeps;
        b->g_xevery = xevery;
    }
    // patch the sweep counter (argument 3 of pt_sweep_kernel) and replay
    cudaKernelNodeParams kp;
    BK(cudaGraphKernelNodeGetParams(b->knode, &kp), "kernel node params");
    uint32_t sweep0 = (uint32_t)b->sweep;
    void* args[8];
    for (int i = 0; i < 8; ++i) args[i] = kp.kernelParams[i];
    args[3] = &sweep0;
    kp.kernelParams = args;
    BK(cudaGraphExecKernelNodeSetParams(b->exec, b->knode, &kp), "patch kernel node");
    BK(cudaGraphLaunch(b->exec, b->stream), "graph launch");
    b->launches += 1;
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
            if (x.J[e] < -3 || x.J[e] > 3) { b->err = "instance " + std::to_string(i) + ": coupler outside [-3, 3]"; return bail(PT_ERR_ARG); }
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
        Tables tb;
        std::string why = build_tables(x.n_temps, x.betas, tb);
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
        thrs += (size_t)b->NT[i] * KT;
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
    BKC(balloc(&b->d_queue, 1), "cudaMalloc queue");
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
    for (auto& kv : b->sched) kv.second = ShapeSched();
    for (int i = 0; i < n_inst; ++i) b->sched[b->L[i]];
    for (auto& kv : b->sched) default_shape_sched(kv.first, max_temps_of(b, kv.first), n_runs, b->block, false, kv.second);
    BKC(cudaMemcpy(b->d_desc, b->desc.data(), sizeof(InstDesc) * b->desc.size(), cudaMemcpyHostToDevice), "upload desc");
    BKC(cudaMemcpy(b->d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice), "upload items");
    // per-L smem check against the largest temperature count of that L
    int rc = build_bundles(b);
    if (rc) return bail(rc);
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
    cudaFree(b->spins); cudaFree(b->E); cudaFree(b->perm); cudaFree(b->best); cudaFree(b->first);
    cudaFree(b->macc); cudaFree(b->xacc); cudaFree(b->jw); cudaFree(b->thr); cudaFree(b->xoff);
    cudaFree(b->xthr); cudaFree(b->xhint); cudaFree(b->nbr); cudaFree(b->d_desc); cudaFree(b->d_items);
    cudaFree(b->d_bundles); cudaFree(b->d_queue); cudaFree(b->d_tts);
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
    if (block > 0 && (block % 32 != 0 || block > MAX_THREADS))
        return bfail(b, PT_ERR_ARG, "block must be a multiple of 32, <= 1024");
    if (chimera_L > 0 && !b->sched.count(chimera_L)) return bfail(b, PT_ERR_ARG, "no instance of that size");
    // validate on copies; the batch changes only when everything fits
    const int nblock = block > 0 ? block : b->block;
    std::map<int, ShapeSched> sched = b->sched;
    if (chimera_L > 0) {
        ShapeSched s = sched[chimera_L];
        s.sp = slot_parallel;
        s.ipc = std::min<int>(runs_per_cta, b->R);
        const int tpr = sched_threads(chimera_L, s);
        if (slot_parallel < 1 || runs_per_cta < 1 || tpr < 32 || tpr * s.ipc > nblock)
            return bfail(b, PT_ERR_ARG, "need threads per run >= 32 and threads per run * runs_per_cta <= block");
        if (s.team == 0 && tpr % 32 != 0)
            return bfail(b, PT_ERR_ARG, "cell-major: slot_parallel * L^2 must be a multiple of 32");
        sched[chimera_L] = s;
    }
    for (auto& kv : sched)           // keep every size inside the block
        if (sched_threads(kv.first, kv.second) * kv.second.ipc > nblock)
            default_shape_sched(kv.first, max_temps_of(b, kv.first), b->R, nblock, b->slot_major, kv.second);
    const std::map<int, ShapeSched> old_sched = b->sched;
    const int old_block = b->block;
    b->sched = sched;
    b->block = nblock;
    int rc = build_bundles(b);
    if (rc) {
        b->sched = old_sched;
        b->block = old_block;
        return rc;
    }
    BK(cudaStreamSynchronize(b->stream), "sync schedule");
    return PT_OK;
}

int pt_batch_set_mapping(pt_batch* b, int32_t chimera_L, int32_t team, int32_t slot_parallel, int32_t runs_per_cta)
{
    if (!b || team < 0) return bfail(b, PT_ERR_ARG, "team must be >= 0");
    if (team > 0 && (team > 32 || (team & (team - 1)) != 0))
        return bfail(b, PT_ERR_ARG, "team must be a power of two <= 32");
    if (chimera_L > 0 && !b->sched.count(chimera_L)) return bfail(b, PT_ERR_ARG, "no instance of that size");
    // validate on copies; the batch changes only when everything fits
    const bool sm = team > 0;
    std::map<int, ShapeSched> sched = b->sched;
    if (sm != b->slot_major)        // the other sizes follow to the new mapping
        for (auto& kv : sched)
            default_shape_sched(kv.first, max_temps_of(b, kv.first), b->R, b->block, sm, kv.second);
    if (chimera_L > 0) {
        ShapeSched s = sched[chimera_L];
        s.team = team;
        if (slot_parallel > 0) s.sp = slot_parallel;
        if (runs_per_cta > 0) s.ipc = std::min<int>(runs_per_cta, b->R);
        const int tpr = sched_threads(chimera_L, s);
        if (tpr < 32 || tpr * s.ipc > b->block || (!sm && tpr % 32 != 0))
            return bfail(b, PT_ERR_ARG, "mapping does not fit the block (threads per run >= 32, x runs_per_cta <= block)");
        if (bundle_smem_bytes(chimera_L, max_temps_of(b, chimera_L), s.ipc, team) > 227 * 1024)
            return bfail(b, PT_ERR_ARG, "shared memory above 227 KB");
        sched[chimera_L] = s;
    }
    const std::map<int, ShapeSched> old_sched = b->sched;
    const bool old_sm = b->slot_major;
    b->sched = sched;
    b->slot_major = sm;
    int rc = build_bundles(b);
    if (rc) {
        b->sched = old_sched;
        b->slot_major = old_sm;
        return rc;
    }
    BK(cudaStreamSynchronize(b->stream), "sync mapping");
    return PT_OK;
}

int pt_batch_get_schedule(const pt_batch* b, int32_t chimera_L, int32_t* block, int32_t* slot_parallel,
                          int32_t* runs_per_cta)
{
    if (!b) return PT_ERR_ARG;
    if (block) *block = b->block;
    auto it = b->sched.find(chimera_L);
    if (it == b->sched.end()) return PT_ERR_ARG;
    if (slot_parallel) *slot_parallel = it->second.sp;
    if (runs_per_cta) *runs_per_cta = it->second.ipc;
    return PT_OK;
}

int pt_batch_get_mapping(const pt_batch* b, int32_t chimera_L, int32_t* team)
{
    if (!b) return PT_ERR_ARG;
    auto it = b->sched.find(chimera_L);
    if (it == b->sched.end()) return PT_ERR_ARG;
    if (team) *team = b->slot_major ? it->second.team : 0;
    return PT_OK;
}

// Times candidate schedules and keeps the fastest.  For each block size in
// {256, 512}, each mapping (cell-major, slot-major) and each Chimera size,
// every schedule that fits is timed on all instances of that size for
// `trial_sweeps` sweeps; the (block, mapping) whose best per-size schedules
// give the shortest predicted batch time wins.  The state is reset afterwards.
int pt_batch_autotune(pt_batch* b, int32_t trial_sweeps, int32_t* block_out)
{
    if (!b || trial_sweeps < 1) return bfail(b, PT_ERR_ARG, "need trial_sweeps >= 1");
    std::map<int, int64_t> work;          // attempts per sweep per size
    std::map<int, int> maxnt;
    for (int i = 0; i < b->n_inst; ++i) {
        work[b->L[i]] += (int64_t)b->R * b->NT[i] * b->N[i];
        maxnt[b->L[i]] = std::max(maxnt[b->L[i]], b->NT[i]);
    }
    const int old_block = b->block;
    const bool old_sm = b->slot_major;
    const std::map<int, ShapeSched> old_sched = b->sched;
    auto restore = [&]() {
        b->block = old_block;
        b->slot_major = old_sm;
        b->sched = old_sched;
        build_bundles(b);
    };
    double best_total = 1e300;
    int best_block = b->block;
    bool best_sm = b->slot_major;
    std::map<int, ShapeSched> best_sched = b->sched;
    for (int block : {256, 512}) {
        for (bool sm : {false, true}) {
            b->block = block;
            b->slot_major = sm;
            std::map<int, ShapeSched> chosen;
            double total = 0.0;
            for (auto& kv : work) {
                const int L = kv.first, L2 = L * L, NT = maxnt[L];
                // (team, slot_parallel) candidates of this mapping
                std::vector<std::pair<int, int>> cands;
                if (!sm) {
                    for (int sp : {1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64})
                        if (sp <= NT && sp * L2 <= block && (sp * L2) % 32 == 0) cands.push_back({0, sp});
                } else {
                    for (int team : {2, 4, 8, 16, 32}) {
                        if (team > 2 * L2 && !cands.empty()) break;
                        int prev = 0;
                        for (int nt : {NT, (NT + 1) / 2, (NT + 3) / 4, (NT + 7) / 8})
                            if (nt != prev && nt * team >= 32 && nt * team <= block) {
                                cands.push_back({team, nt});
                                prev = nt;
                            }
                    }
                }
                double best_rate = 0.0;
                ShapeSched bs;
                for (const auto& c : cands) {
                    const int tpr = c.first > 0 ? c.second * c.first : c.second * L2;
                    for (int ipc : {1, 2, 4, 8, 16}) {
                        if (tpr * ipc > block || ipc > b->R) break;
                        if (bundle_smem_bytes(L, NT, ipc, c.first) > 200 * 1024) break;
                        ShapeSched& s = b->sched[L];
                        s.team = c.first;
                        s.sp = c.second;
                        s.ipc = ipc;
                        std::vector<int> only{L};
                        int rc = build_bundles(b, &only, 0);
                        if (rc) continue;
                        int64_t att = 0;
                        for (const Bundle& x : b->bundles) att += (int64_t)x.nitems * b->NT[x.inst] * b->N[x.inst];
                        att *= trial_sweeps;
                        cudaError_t e = cudaEventRecord(b->e0, b->stream);
                        if (e == cudaSuccess) e = cudaMemsetAsync(b->d_queue, 0, sizeof(int), b->stream);
                        if (e == cudaSuccess)
                            e = launch_sweeps(b->d_desc, b->d_bundles, (int)b->bundles.size(), b->grid, b->block,
                                              b->smem, 0u, trial_sweeps, 1, 0, b->d_queue, b->stream, sm);
                        if (e == cudaSuccess) e = cudaEventRecord(b->e1, b->stream);
                        if (e == cudaSuccess) e = cudaEventSynchronize(b->e1);
                        float ms = 0.f;
                        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, b->e0, b->e1);
                        if (e != cudaSuccess) {
                            const int code = bcuda(b, e, "trial launch");
                            restore();
                            return code;
                        }
                        const double rate = att / (ms * 1e-3);
                        if (rate > best_rate) { best_rate = rate; bs = s; }
                    }
                }
                if (best_rate <= 0.0) { total = 1e300; break; }
                chosen[L] = bs;
                total += (double)kv.second / best_rate;
            }
            if (total < best_total) { best_total = total; best_block = block; best_sm = sm; best_sched = chosen; }
        }
    }
    b->block = best_block;
    b->slot_major = best_sm;
    for (auto& kv : best_sched) b->sched[kv.first] = kv.second;
    int rc = build_bundles(b);
    if (rc) { restore(); return rc; }
    rc = pt_batch_reset(b);
    if (rc) return rc;
    if (block_out) *block_out = b->block;
    return PT_OK;
}

int pt_batch_info(const pt_batch* b, double* last_run_ms, int32_t* grid, int32_t* block, int32_t* n_bundles,
                  uint64_t* launches)
{
    if (!b) return PT_ERR_ARG;
    if (last_run_ms) *last_run_ms = b->last_ms;
    if (grid) *grid = b->grid;
    if (block) *block = b->block;
    if (n_bundles) *n_bundles = (int32_t)b->bundles.size();
    if (launches) *launches = b->launches;
    return PT_OK;
}

}  // extern "C"
