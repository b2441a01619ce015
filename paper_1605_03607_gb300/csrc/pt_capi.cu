// pt_capi.cu -- host runtime and C ABI (include/pt.h) of the GB300 PT engine.
//
// The host side does only what has to happen on the host: argument checks,
// FP64 acceptance tables (the Metropolis rule of Sec. II and the exchange rule
// with detailed balance), repacking the couplers into the kernels' layout,
// the random draws of Algorithm 1 (one Philox4x32-10 call per step), and the
// accept/reject bookkeeping of the engineering loop.  Every sweep, energy and
// TTS reduction runs in the kernels of pt_kernels.cu.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/pt.h"
#include "pt_internal.h"
#include "pt_host.h"
#include "pt_kernels.h"

using namespace ptg;

namespace {

std::mutex g_err_mu;
std::string g_create_err = "no error";

// A set of instances of one shape (L, NT, R) sharing one ladder.
struct Group {
    int L = 0, NT = 0, R = 0, n_inst = 0;
    int8_t* spins = nullptr;
    int32_t* E = nullptr;
    uint8_t* perm = nullptr;
    int32_t *best = nullptr, *first = nullptr;
    unsigned long long *macc = nullptr, *xacc = nullptr;
    uint32_t* jw = nullptr;          // [n_inst][L2][2][8]
    InstDesc* d_desc = nullptr;
    int2* d_items = nullptr;
    Bundle* d_bundles = nullptr;
    Bundle* d_sub = nullptr;         // a subset of the bundles (doubling budget: undecided instances)
    int32_t* d_tts = nullptr;        // [n_inst][3]
    int32_t* d_targets = nullptr;    // [n_inst] per-instance TTS targets (LAO)
    int* d_queue = nullptr;
    std::vector<InstDesc> desc;
    std::vector<Bundle> bundles;
    int block = 0, smem = 0;
    uint64_t sweep = 0;
    // temperature random walk (main group only, when tracked)
    bool walk = false;
    unsigned long long *whot = nullptr, *wtrips = nullptr;
    uint8_t* wstate = nullptr;
    uint64_t walk_passes = 0;        // exchange passes since the counters were cleared
};

}  // namespace

struct pt_handle {
    int L = 0, NT = 0, R = 0, N = 0, n_edges = 0;
    uint32_t seed = 0, uid = 0;
    std::vector<int8_t> J;
    std::vector<double> betas;
    Tables tb;
    int kt = KT_DEFAULT;       // Metropolis table rows per slot (grows with the couplers, ensure_table_rows)
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // device tables shared by every group of this handle
    uint32_t* d_thr = nullptr;
    int32_t* d_xoff = nullptr;
    uint32_t* d_xthr = nullptr;
    float* d_xhint = nullptr;
    int16_t* d_nbr = nullptr;
    Group main, cand;
    int sp = 0, ipc = 0, spl = 4096;
    int team = 0;              // 0: cell-major mapping; > 0: slot-major with teams of this size
    uint64_t launches = 0;
    // timing of sweep launches
    bool timing = false;
    std::vector<cudaEvent_t> ev;
    int ev_used = 0;
    double last_ms = 0.0;
    int last_launches = 0;
    double total_ms = 0.0;
    uint64_t total_launches = 0;
    // evaluation accounting (every batched PT-TTS evaluation)
    uint64_t evals = 0, batches = 0;
    double eval_ms = 0.0;
    cudaEvent_t eb0 = nullptr, eb1 = nullptr;
    // loop adaptive optimisation (planted instance)
    bool lao = false;
    uint32_t lao_uid = 0;
    int lao_w_max = 3;
    std::vector<int8_t> planted;
    std::vector<int32_t> loops;      // [n_loops][PT_LOOP_WORDS]
    int32_t E_gs = 0;
    // engineering loop
    bool eng = false;
    pt_rule rule{};
    uint32_t base_uid = 0;
    int32_t tts_cur = 0;
    int32_t hits_cur = 0;      // runs that reached the target in the current instance's evaluation
    // adaptive budget of Appendix B (engineer_set_adaptive): runs per evaluation
    bool adapt = false;
    int32_t n_cur = 0, n_min = 0;
    int64_t cost_max = 0;
    double beta_per_run = 0.0;
    std::vector<int32_t> last_levels;   // deciding levels of the last doubling evaluation of candidates
    // Evaluated candidates of RAO steps past the end of the last engineer_run call (each batch is
    // evaluated in full, spec candidates), kept with everything their evaluation depends on; the
    // next call uses them only if it starts at `step` and all of it is unchanged.
    struct SpecCache {
        bool valid = false;
        uint32_t step = 0;             // RAO step of entry 0
        int32_t n_runs = 0;
        uint32_t base_uid = 0;
        pt_rule rule{};
        std::vector<int8_t> J;
        std::vector<int32_t> e, v, res, level;   // res: tts, hits, target per entry
        std::vector<uint32_t> cu, ua;
    } spec_cache;
    // The same for lao_run: candidates also depend on the loop list and E_GS, and an accepted one
    // replaces the couplers and one loop record.
    struct LaoCache {
        bool valid = false;
        uint32_t step = 0;
        pt_rule rule{};
        std::vector<int8_t> J;
        std::vector<int32_t> loops;
        int32_t E_gs = 0;
        std::vector<int8_t> Jc;                        // candidates' couplers [count][n_edges]
        std::vector<int32_t> rem, egs, recs, res;      // recs [count][PT_LOOP_WORDS], res 3 per entry
        std::vector<uint32_t> cu, ua;
    } lao_cache;
    std::string err = "no error";
};

namespace {

int fail(pt_handle* h, int code, const std::string& msg)
{
    if (h) h->err = msg;
    else {
        std::lock_guard<std::mutex> g(g_err_mu);
        g_create_err = msg;
    }
    return code;
}

int cuda_fail(pt_handle* h, cudaError_t e, const char* what)
{
    return fail(h, e == cudaErrorMemoryAllocation ? PT_ERR_OOM : PT_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call, what)                                        \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, what); \
    } while (0)

template <class T>
cudaError_t dalloc(T** p, size_t n)
{
    return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (n ? n : 1));
}

void free_group(Group& g)
{
    cudaFree(g.spins); cudaFree(g.E); cudaFree(g.perm); cudaFree(g.best); cudaFree(g.first);
    cudaFree(g.macc); cudaFree(g.xacc); cudaFree(g.jw); cudaFree(g.d_desc); cudaFree(g.d_items);
    cudaFree(g.d_bundles); cudaFree(g.d_sub); cudaFree(g.d_tts); cudaFree(g.d_queue);
    cudaFree(g.whot); cudaFree(g.wtrips); cudaFree(g.wstate); cudaFree(g.d_targets);
    g = Group();
}

// A doubling budget S0, 2 S0, ... Smax: Smax = S0 * 2^k, Smax <= 2^30 (pass_mult 1).
bool doubling_ok(int32_t S0, int32_t Smax, int32_t pass_mult)
{
    if (S0 < 1 || Smax < S0 || Smax > (1 << 30) || pass_mult != 1) return false;
    int64_t x = S0;
    while (x < Smax) x *= 2;
    return x == Smax;
}

// Default schedule: about 256 threads per run, a multiple of 32.
void default_schedule(int L, int NT, int R, int& sp, int& ipc, int kt)
{
    const int L2 = L * L;
    sp = std::max(1, 256 / L2);
    if (sp > NT) sp = NT;
    while ((sp * L2) % 32 != 0) ++sp;
    const int tpi = sp * L2;
    ipc = std::max(1, 512 / tpi);
    if (ipc > R) ipc = R;
    while (ipc > 1 && bundle_smem_bytes(L, NT, ipc, 0, false, kt) > 110 * 1024) --ipc;
}

int check_schedule(pt_handle* h, int L, int NT, int sp, int ipc, int team)
{
    const int L2 = L * L;
    if (sp < 1 || ipc < 1) return fail(h, PT_ERR_ARG, "schedule values must be >= 1");
    if (team > 0) {
        if (team > 32 || (team & (team - 1)) != 0) return fail(h, PT_ERR_ARG, "team must be a power of two <= 32");
        if (sp * team < 32) return fail(h, PT_ERR_ARG, "teams * team must be >= 32");
        if (sp * team * ipc > MAX_THREADS_SM)
            return fail(h, PT_ERR_ARG, "more than 768 threads per CTA (slot-major mapping)");
    } else {
        if ((sp * L2) % 32 != 0) return fail(h, PT_ERR_ARG, "slot_parallel * L^2 must be a multiple of 32");
        if (sp * L2 * ipc > MAX_THREADS) return fail(h, PT_ERR_ARG, "more than 1024 threads per CTA");
    }
    if (bundle_smem_bytes(L, NT, ipc, team, h->main.walk, h->kt) > 227 * 1024)
        return fail(h, PT_ERR_ARG, "shared memory above 227 KB");
    return PT_OK;
}

int group_alloc(pt_handle* h, Group& g, int n_inst)
{
    g.L = h->L; g.NT = h->NT; g.R = h->R; g.n_inst = n_inst;
    const size_t reps = (size_t)n_inst * h->R * h->NT;
    const size_t runs = (size_t)n_inst * h->R;
    const size_t npair = (size_t)(h->NT > 1 ? h->NT - 1 : 1);
    CK(dalloc(&g.spins, reps * h->N), "cudaMalloc spins");
    CK(dalloc(&g.E, reps), "cudaMalloc E");
    CK(dalloc(&g.perm, reps), "cudaMalloc perm");
    CK(dalloc(&g.best, runs), "cudaMalloc best");
    CK(dalloc(&g.first, runs), "cudaMalloc first");
    CK(dalloc(&g.macc, reps), "cudaMalloc macc");
    CK(dalloc(&g.xacc, runs * npair), "cudaMalloc xacc");
    CK(dalloc(&g.jw, (size_t)n_inst * h->L * h->L * 16), "cudaMalloc jw");
    CK(dalloc(&g.d_desc, (size_t)n_inst), "cudaMalloc desc");
    CK(dalloc(&g.d_items, runs), "cudaMalloc items");
    CK(dalloc(&g.d_tts, (size_t)n_inst * 3), "cudaMalloc tts");
    CK(dalloc(&g.d_targets, (size_t)n_inst), "cudaMalloc targets");
    CK(dalloc(&g.d_queue, 1), "cudaMalloc queue");
    g.desc.resize(n_inst);
    for (int i = 0; i < n_inst; ++i) {
        InstDesc& d = g.desc[i];
        const size_t r0 = (size_t)i * h->R;
        d.L = h->L; d.NT = h->NT; d.R = h->R; d.n_xpairs = h->NT - 1;
        d.seed = h->seed; d.uid = h->uid;
        d.kt = h->kt;
        d.jw = g.jw + (size_t)i * h->L * h->L * 16;
        d.nbr = h->d_nbr; d.thr = h->d_thr; d.xoff = h->d_xoff; d.xthr = h->d_xthr; d.xhint = h->d_xhint;
        d.spins = g.spins + r0 * h->NT * h->N;
        d.E = g.E + r0 * h->NT;
        d.perm = g.perm + r0 * h->NT;
        d.best = g.best + r0;
        d.first = g.first + r0;
        d.macc = g.macc + r0 * h->NT;
        d.xacc = g.xacc + r0 * npair;
    }
    std::vector<int2> items(runs);
    for (int i = 0; i < n_inst; ++i)
        for (int r = 0; r < h->R; ++r) items[(size_t)i * h->R + r] = make_int2(i, r);
    CK(cudaMemcpyAsync(g.d_items, items.data(), sizeof(int2) * runs, cudaMemcpyHostToDevice, h->stream), "upload items");
    return PT_OK;
}

// The new bundle list replaces the group's only when every step succeeded, so
// a failure leaves the previous schedule in place and launchable.
int group_schedule(pt_handle* h, Group& g)
{
    std::vector<Bundle> bundles;
    const int L2 = g.L * g.L;
    for (int i = 0; i < g.n_inst; ++i)
        for (int r = 0; r < g.R; r += h->ipc) {
            Bundle b;
            b.inst = i; b.run0 = r; b.nitems = std::min(h->ipc, g.R - r); b.sp = h->sp; b.team = h->team;
            bundles.push_back(b);
        }
    const int block = (h->team > 0 ? h->sp * h->team : h->sp * L2) * h->ipc;
    const int smem = (int)bundle_smem_bytes(g.L, g.NT, h->ipc, h->team, g.walk, h->kt);
    int cap = 0;
    CK(sweep_smem_capacity(&cap), "shared memory capacity");
    if (smem > cap) return fail(h, PT_ERR_ARG, "bundle needs more shared memory than a CTA can have");
    CK(set_sweep_smem_limit(cap), "cudaFuncSetAttribute");
    Bundle* d = nullptr;
    Bundle* dsub = nullptr;
    CK(dalloc(&d, bundles.size()), "cudaMalloc bundles");
    cudaError_t e = dalloc(&dsub, bundles.size());
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d, bundles.data(), sizeof(Bundle) * bundles.size(), cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) {
        cudaFree(d);
        cudaFree(dsub);
        return cuda_fail(h, e, "upload bundles");
    }
    cudaFree(g.d_bundles);
    cudaFree(g.d_sub);
    g.d_sub = dsub;               // room for any subset of the full list
    g.d_bundles = d;
    g.bundles.swap(bundles);
    g.block = block;
    g.smem = smem;
    return PT_OK;
}

int upload_desc(pt_handle* h, Group& g)
{
    CK(cudaMemcpyAsync(g.d_desc, g.desc.data(), sizeof(InstDesc) * g.desc.size(),
                       cudaMemcpyHostToDevice, h->stream), "upload desc");
    return PT_OK;
}

int upload_couplers(pt_handle* h, Group& g, int inst, const int8_t* J)
{
    std::vector<uint32_t> jw((size_t)h->L * h->L * 16);
    pack_couplers(h->L, J, jw.data());
    CK(cudaMemcpyAsync(g.jw + (size_t)inst * jw.size(), jw.data(), sizeof(uint32_t) * jw.size(),
                       cudaMemcpyHostToDevice, h->stream), "upload couplers");
    // the pageable source must stay alive until the copy is done
    CK(cudaStreamSynchronize(h->stream), "sync after coupler upload");
    return PT_OK;
}

// Zeroes the walk counters and states of a tracked group.
int walk_clear(pt_handle* h, Group& g)
{
    if (!g.walk) return PT_OK;
    const size_t reps = (size_t)g.n_inst * g.R * g.NT;
    CK(cudaMemsetAsync(g.whot, 0, 8 * reps, h->stream), "clear walk");
    CK(cudaMemsetAsync(g.wtrips, 0, 8 * reps, h->stream), "clear walk");
    CK(cudaMemsetAsync(g.wstate, 0, reps, h->stream), "clear walk");
    g.walk_passes = 0;
    return PT_OK;
}

int group_reset(pt_handle* h, Group& g, bool draw)
{
    int rc = walk_clear(h, g);
    if (rc) return rc;
    CK(launch_init(g.d_desc, g.d_items, g.n_inst * g.R, draw, h->stream), "init kernel");
    CK(launch_energy(g.d_desc, g.d_items, g.n_inst * g.R, 0, h->stream), "energy kernel");
    h->launches += 2;
    g.sweep = 0;
    return PT_OK;
}

int ensure_events(pt_handle* h, int n)
{
    while ((int)h->ev.size() < n) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e), "cudaEventCreate");
        h->ev.push_back(e);
    }
    return PT_OK;
}

int group_sweeps(pt_handle* h, Group& g, int64_t n, int xevery, const Bundle* dsub = nullptr, int nsub = 0)
{
    const Bundle* db = dsub ? dsub : g.d_bundles;
    const int nb = dsub ? nsub : (int)g.bundles.size();
    const int nl = (int)((n + h->spl - 1) / h->spl);
    if (h->timing) {
        int rc = ensure_events(h, 2 * nl);
        if (rc) return rc;
    }
    int64_t done = 0;
    int li = 0;
    while (done < n) {
        const int chunk = (int)std::min<int64_t>(h->spl, n - done);
        if (h->timing) CK(cudaEventRecord(h->ev[2 * li], h->stream), "event");
        CK(launch_sweeps(g.d_desc, db, nb, nb, g.block, g.smem, (uint32_t)g.sweep, chunk, xevery, 0, nullptr,
                         h->stream, h->team > 0, g.walk, g.L),
           "sweep kernel");
        if (g.walk && g.NT > 1 && xevery > 0)
            g.walk_passes += (g.sweep + chunk) / (uint64_t)xevery - g.sweep / (uint64_t)xevery;
        if (h->timing) CK(cudaEventRecord(h->ev[2 * li + 1], h->stream), "event");
        ++h->launches;
        ++li;
        g.sweep += (uint64_t)chunk;
        done += chunk;
    }
    h->ev_used = h->timing ? li : 0;
    h->last_launches = li;
    return PT_OK;
}

int collect_timing(pt_handle* h)
{
    if (!h->timing) return PT_OK;
    CK(cudaStreamSynchronize(h->stream), "sync for timing");
    double ms = 0.0;
    for (int i = 0; i < h->ev_used; ++i) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, h->ev[2 * i], h->ev[2 * i + 1]), "event time");
        ms += t;
    }
    h->last_ms = ms;
    h->total_ms += ms;
    h->total_launches += (uint64_t)h->ev_used;
    return PT_OK;
}

int group_tts(pt_handle* h, Group& g, int32_t target, int32_t horizon, std::vector<int32_t>& out)
{
    CK(launch_tts(g.d_desc, g.n_inst, target, horizon, g.d_tts, h->stream), "tts kernel");
    ++h->launches;
    out.assign((size_t)g.n_inst * 3, 0);
    CK(cudaMemcpyAsync(out.data(), g.d_tts, sizeof(int32_t) * out.size(), cudaMemcpyDeviceToHost,
                       h->stream), "download tts");
    CK(cudaStreamSynchronize(h->stream), "sync tts");
    return PT_OK;
}

// Full evaluation of every instance of g: fresh runs, pass_mult*S sweeps, TTS at horizon S.
// targets (host, one per instance, may be NULL): per-instance TTS targets.
int group_eval(pt_handle* h, Group& g, int32_t S, int32_t pass_mult, int32_t xevery,
               std::vector<int32_t>& out, int32_t target = PT_TARGET_BEST, const int32_t* targets = nullptr,
               const Bundle* dsub = nullptr, int nsub = 0)
{
    int rc;
    if (!h->eb0) {
        CK(cudaEventCreate(&h->eb0), "cudaEventCreate");
        CK(cudaEventCreate(&h->eb1), "cudaEventCreate");
    }
    if ((rc = upload_desc(h, g))) return rc;
    CK(cudaEventRecord(h->eb0, h->stream), "event");
    if ((rc = group_reset(h, g, true))) return rc;
    if ((rc = group_sweeps(h, g, (int64_t)S * pass_mult, xevery, dsub, nsub))) return rc;
    if (targets)
        CK(cudaMemcpyAsync(g.d_targets, targets, sizeof(int32_t) * g.n_inst, cudaMemcpyHostToDevice, h->stream),
           "upload targets");
    CK(launch_tts(g.d_desc, g.n_inst, target, S, g.d_tts, h->stream, targets ? g.d_targets : nullptr),
       "tts kernel");
    ++h->launches;
    CK(cudaEventRecord(h->eb1, h->stream), "event");
    out.assign((size_t)g.n_inst * 3, 0);
    CK(cudaMemcpyAsync(out.data(), g.d_tts, sizeof(int32_t) * out.size(), cudaMemcpyDeviceToHost,
                       h->stream), "download tts");
    CK(cudaStreamSynchronize(h->stream), "sync eval");
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->eb0, h->eb1), "event time");
    h->eval_ms += ms;
    h->evals += (uint64_t)g.n_inst;
    h->batches += 1;
    return collect_timing(h);
}

// Evaluation of every instance of g under the doubling budget: fresh runs,
// then levels S0, 2 S0, ... Smax on the same runs.  After each level the TTS
// of every instance is taken against its best energy within that level
// (horizon = level); an instance is decided at the first level with
// TTS <= level / 4, and later levels sweep only the undecided instances'
// bundles.  Unsolved after Smax: TTS = Smax + 1.  out = n_inst x {tts, hits,
// target}; levels = the deciding level of each instance.
int group_eval_doubling(pt_handle* h, Group& g, int32_t S0, int32_t Smax, int32_t xevery, std::vector<int32_t>& out,
                        std::vector<int32_t>& levels)
{
    int rc;
    if (!h->eb0) {
        CK(cudaEventCreate(&h->eb0), "cudaEventCreate");
        CK(cudaEventCreate(&h->eb1), "cudaEventCreate");
    }
    if ((rc = upload_desc(h, g))) return rc;
    CK(cudaEventRecord(h->eb0, h->stream), "event");
    if ((rc = group_reset(h, g, true))) return rc;
    const int n = g.n_inst;
    std::vector<char> open((size_t)n, 1);
    out.assign((size_t)n * 3, 0);
    levels.assign((size_t)n, 0);
    std::vector<Bundle> sub;
    std::vector<int32_t> lv_out;
    double ms_total = 0.0;
    for (int64_t lv = S0;; lv *= 2) {
        sub.clear();
        for (const Bundle& b : g.bundles)
            if (b.inst < n && open[(size_t)b.inst]) sub.push_back(b);
        CK(cudaMemcpyAsync(g.d_sub, sub.data(), sizeof(Bundle) * sub.size(), cudaMemcpyHostToDevice, h->stream),
           "upload bundle subset");
        if ((rc = group_sweeps(h, g, lv - (int64_t)g.sweep, xevery, g.d_sub, (int)sub.size()))) return rc;
        if ((rc = group_tts(h, g, PT_TARGET_BEST, (int32_t)lv, lv_out))) return rc;   // synchronises
        if ((rc = collect_timing(h))) return rc;
        if (h->timing) ms_total += h->last_ms;
        bool any = false;
        for (int i = 0; i < n; ++i) {
            if (!open[(size_t)i]) continue;
            const int32_t t = lv_out[(size_t)i * 3];
            const bool last = lv >= Smax;
            if (t <= lv / 4 || last) {
                out[(size_t)i * 3 + 0] = t <= lv / 4 ? t : Smax + 1;
                out[(size_t)i * 3 + 1] = lv_out[(size_t)i * 3 + 1];
                out[(size_t)i * 3 + 2] = lv_out[(size_t)i * 3 + 2];
                levels[(size_t)i] = (int32_t)lv;
                open[(size_t)i] = 0;
            } else {
                any = true;
            }
        }
        if (!any) break;
    }
    CK(cudaEventRecord(h->eb1, h->stream), "event");
    CK(cudaEventSynchronize(h->eb1), "sync eval");
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->eb0, h->eb1), "event time");
    h->eval_ms += ms;
    h->evals += (uint64_t)n;
    h->batches += 1;
    if (h->timing) h->last_ms = ms_total;
    return PT_OK;
}

// Draw of proposal j for step t against couplers J (Algorithm 1, one perturbed edge).
void engineer_draw(const pt_handle* h, const int8_t* J, uint32_t step, uint32_t proposal,
                   int32_t& edge, int32_t& value, uint32_t& uid, uint32_t& uacc)
{
    static const int8_t vals[6] = {-3, -2, -1, 1, 2, 3};
    const uint32_t ctr[4] = {step, proposal, 0u, 3u};
    uint32_t w[4];
    philox_host(ctr, h->seed, h->base_uid, w);
    edge = (int32_t)(((uint64_t)w[0] * (uint64_t)h->n_edges) >> 32);
    const int pick = (int)(((uint64_t)w[1] * 5u) >> 32);
    int n = 0;
    value = 0;
    for (int a = 0; a < 6; ++a) {
        if (vals[a] == J[edge]) continue;
        if (n == pick) value = vals[a];
        ++n;
    }
    uid = w[2];
    uacc = w[3];
}

bool engineer_accept(const pt_rule& rule, int32_t cur, int32_t cand, uint32_t uacc)
{
    const int64_t gain = (int64_t)rule.direction * ((int64_t)cand - (int64_t)cur);
    if (gain > 0) return true;
    if (rule.beta_rao >= 0.0) {
        const double dt = std::fabs((double)cand - (double)cur);
        return uacc < to_u32_threshold(std::exp(-rule.beta_rao * dt));
    }
    return false;
}

int ensure_candidates(pt_handle* h, int k);
int ensure_table_rows(pt_handle* h, int kmax);

// PT-TTS evaluation of k candidate coupler vectors (host [k][n_edges]) with
// PT keys uids[0..k-1], as one batched launch sequence; res = k x {tts, hits, target}.
int eval_candidates(pt_handle* h, int k, const int8_t* Jc, const uint32_t* uids, std::vector<int32_t>& res,
                    int32_t target = PT_TARGET_BEST, const int32_t* targets = nullptr, int n_eval = 0)
{
    int rc = ensure_candidates(h, k);
    if (rc) return rc;
    int kmax = 0;
    for (int j = 0; j < k; ++j) kmax = std::max(kmax, coupler_kmax(h->L, Jc + (size_t)j * h->n_edges));
    if ((rc = ensure_table_rows(h, kmax))) return rc;
    Group& g = h->cand;
    std::vector<uint32_t> jw((size_t)k * h->L * h->L * 16);
    for (int j = 0; j < k; ++j) {
        pack_couplers(h->L, Jc + (size_t)j * h->n_edges, jw.data() + (size_t)j * h->L * h->L * 16);
        g.desc[j].uid = uids[j];
    }
    CK(cudaMemcpyAsync(g.jw, jw.data(), 4 * jw.size(), cudaMemcpyHostToDevice, h->stream), "upload candidates");
    // evaluate only the first k candidates, with their first n_eval runs
    // (all runs when n_eval is 0): shrink the group view temporarily
    const int nr = (n_eval > 0 && n_eval < h->R) ? n_eval : h->R;
    const int n_full = g.n_inst;
    std::vector<Bundle> keep = g.bundles;
    g.n_inst = k;
    std::vector<Bundle> sub;
    for (Bundle b : keep) {
        if (b.inst >= k || b.run0 >= nr) continue;
        b.nitems = std::min(b.nitems, nr - b.run0);
        sub.push_back(b);
    }
    g.bundles = sub;
    for (int j = 0; j < k; ++j) g.desc[j].R = nr;            // the TTS reduction's run count
    if (h->rule.max_sweeps > 0 && !targets && target == PT_TARGET_BEST) {
        rc = group_eval_doubling(h, g, h->rule.S, h->rule.max_sweeps, h->rule.exchange_every, res, h->last_levels);
    } else {
        rc = cudaMemcpyAsync(g.d_sub, sub.data(), sizeof(Bundle) * sub.size(), cudaMemcpyHostToDevice, h->stream)
                 == cudaSuccess ? PT_OK : fail(h, PT_ERR_CUDA, "upload bundle subset");
        if (!rc)
            rc = group_eval(h, g, h->rule.S, h->rule.pass_mult, h->rule.exchange_every, res, target, targets,
                            g.d_sub, (int)sub.size());
        h->last_levels.assign((size_t)k, h->rule.S * h->rule.pass_mult);
    }
    for (int j = 0; j < k; ++j) g.desc[j].R = h->R;
    g.n_inst = n_full;
    g.bundles = keep;
    return rc;
}

int ensure_candidates(pt_handle* h, int k)
{
    if (h->cand.n_inst >= k) return PT_OK;
    free_group(h->cand);
    int rc = group_alloc(h, h->cand, k);
    if (!rc) rc = group_schedule(h, h->cand);
    // a half-built group (n_inst already set, some buffers missing) must not
    // pass the size check above on a later call
    if (rc) free_group(h->cand);
    return rc;
}

// ------------------------------------------------ planted instances, LAO
// Chimera adjacency with every vertex's neighbours in ascending order (the
// order the loop walks index into) and the edge index of each neighbour.
struct LaoGraph {
    int N = 0, E = 0;
    std::vector<int32_t> ei, ej;
    std::vector<std::array<int, 6>> nb, ne;
    std::vector<int> deg;
    explicit LaoGraph(int L)
    {
        N = 8 * L * L;
        E = n_edges_of(L);
        ei.resize(E); ej.resize(E);
        int e = 0;
        auto sp = [&](int r, int c, int u, int k) { return 8 * (r * L + c) + 4 * u + k; };
        for (int r = 0; r < L; ++r)
            for (int c = 0; c < L; ++c)
                for (int kv = 0; kv < 4; ++kv)
                    for (int kh = 0; kh < 4; ++kh) { ei[e] = sp(r, c, 0, kv); ej[e] = sp(r, c, 1, kh); ++e; }
        for (int r = 0; r + 1 < L; ++r)
            for (int c = 0; c < L; ++c)
                for (int k = 0; k < 4; ++k) { ei[e] = sp(r, c, 0, k); ej[e] = sp(r + 1, c, 0, k); ++e; }
        for (int r = 0; r < L; ++r)
            for (int c = 0; c + 1 < L; ++c)
                for (int k = 0; k < 4; ++k) { ei[e] = sp(r, c, 1, k); ej[e] = sp(r, c + 1, 1, k); ++e; }
        nb.assign(N, {}); ne.assign(N, {}); deg.assign(N, 0);
        std::vector<std::vector<std::pair<int, int>>> adj(N);
        for (int x = 0; x < E; ++x) {
            adj[ei[x]].push_back({ej[x], x});
            adj[ej[x]].push_back({ei[x], x});
        }
        for (int v = 0; v < N; ++v) {
            std::sort(adj[v].begin(), adj[v].end());
            deg[v] = (int)adj[v].size();
            for (int k = 0; k < deg[v]; ++k) { nb[v][k] = adj[v][k].first; ne[v][k] = adj[v][k].second; }
        }
    }
    int edge(int a, int b) const
    {
        for (int k = 0; k < deg[a]; ++k) if (nb[a][k] == b) return ne[a][k];
        return -1;
    }
};

constexpr uint32_t LAO_P4 = 429496730u;      // floor(0.1 * 2^32): length-4 loops, else length 6
constexpr uint32_t LAO_ATTEMPTS = 1u << 16;

uint32_t lao_word(uint32_t seed, uint32_t uid, uint32_t c0, uint32_t c1, uint32_t c2, int w)
{
    const uint32_t ctr[4] = {c0, c1, c2, 4u};
    uint32_t out[4];
    philox_host(ctr, seed, uid, out);
    return out[w];
}

uint32_t mulhi(uint32_t u, uint32_t n) { return (uint32_t)(((uint64_t)u * n) >> 32); }

int loop_term(const LaoGraph& g, const int8_t* planted, const int32_t* rec, int m)
{
    const int e = rec[3 + m];
    return (m == rec[2] ? 1 : -1) * rec[1] * planted[g.ei[e]] * planted[g.ej[e]];
}

void loop_apply(const LaoGraph& g, const int8_t* planted, const int32_t* rec, int8_t* J, int sign)
{
    for (int m = 0; m < rec[0]; ++m) J[rec[3 + m]] = (int8_t)(J[rec[3 + m]] + sign * loop_term(g, planted, rec, m));
}

// Loop (c0, c1) against couplers J: the length is fixed by attempt 0, then
// placements are drawn until one closes a simple cycle without taking a
// coupler outside [-3, 3].  false when none is found.
bool lao_draw_loop(const LaoGraph& g, const int8_t* planted, const int8_t* J, uint32_t seed, uint32_t uid,
                   uint32_t c0, uint32_t c1, int w_max, int32_t* rec)
{
    const int len = lao_word(seed, uid, c0, c1, 0u, 0) < LAO_P4 ? 4 : 6;
    for (uint32_t a = 0; a < LAO_ATTEMPTS; ++a) {
        uint32_t u[16];
        for (int q = 0; q < 4; ++q) {
            const uint32_t ctr[4] = {c0, c1, (a << 2) | (uint32_t)q, 4u};
            philox_host(ctr, seed, uid, u + 4 * q);
        }
        int v[6];
        bool ok = true;
        v[0] = (int)mulhi(u[1], (uint32_t)g.N);
        for (int m = 1; m < len && ok; ++m) {
            const int p = v[m - 1];
            v[m] = g.nb[p][mulhi(u[1 + m], (uint32_t)g.deg[p])];
            for (int q = 0; q < m; ++q) if (v[q] == v[m]) ok = false;
        }
        if (!ok) continue;
        int32_t r[PT_LOOP_WORDS];
        r[0] = len;
        r[1] = 1 + (int)mulhi(u[8], (uint32_t)w_max);
        r[2] = (int)mulhi(u[9], (uint32_t)len);
        for (int m = 0; m < 6; ++m) r[3 + m] = -1;
        for (int m = 0; m < len && ok; ++m) {
            r[3 + m] = g.edge(v[m], v[(m + 1) % len]);
            if (r[3 + m] < 0) ok = false;
        }
        // the engine's bounds: int8 couplers, and every spin's sum of |J| <= 127
        // (its Metropolis table rows); with the paper's weights (1..5, 350
        // loops on C_8) no placement reaches them
        int Jt[6];
        for (int m = 0; m < len && ok; ++m) {
            Jt[m] = J[r[3 + m]] + loop_term(g, planted, r, m);
            if (Jt[m] < -J_ABS_MAX || Jt[m] > J_ABS_MAX) ok = false;
        }
        for (int m = 0; m < len && ok; ++m) {
            const int x = v[m];
            int sum = 0;
            for (int k = 0; k < g.deg[x]; ++k) {
                const int e = g.ne[x][k];
                int val = J[e];
                for (int q = 0; q < len; ++q) if (r[3 + q] == e) val = Jt[q];
                sum += val < 0 ? -val : val;
            }
            if (sum > KT_MAX - 1) ok = false;
        }
        if (!ok) continue;
        std::memcpy(rec, r, sizeof(r));
        return true;
    }
    return false;
}

int32_t loops_gs(const int32_t* loops, int n)
{
    int32_t e = 0;
    for (int m = 0; m < n; ++m) e -= loops[m * PT_LOOP_WORDS + 1] * (loops[m * PT_LOOP_WORDS] - 2);
    return e;
}

// Mapping (team, slot_parallel, runs_per_cta) of every group of the handle.
// On failure the handle keeps its previous mapping: a group whose new bundle
// list could not be built keeps its old one (group_schedule), and the groups
// already switched are switched back.
int apply_schedule(pt_handle* h, int team, int sp, int ipc)
{
    const int ot = h->team, osp = h->sp, oipc = h->ipc;
    h->team = team;
    h->sp = sp;
    h->ipc = std::min(ipc, h->R);
    int rc = group_schedule(h, h->main);
    if (!rc && h->cand.n_inst > 0 && (rc = group_schedule(h, h->cand))) {
        const std::string why = h->err;
        h->team = ot; h->sp = osp; h->ipc = oipc;
        group_schedule(h, h->main);
        h->err = why;
    }
    if (rc) { h->team = ot; h->sp = osp; h->ipc = oipc; }
    return rc;
}

// Makes the handle's Metropolis table cover local fields up to kmax (rows
// 0 .. kmax): a coupler change that raises some spin's sum of |J| above the
// table's last row rebuilds the table with more rows, points every group's
// instances at it and rebuilds their schedules for the larger shared-memory
// footprint.  Tables never shrink, so results do not depend on the order of
// the changes (every row is a function of (beta, k) alone).
int ensure_table_rows(pt_handle* h, int kmax)
{
    if (kmax > KT_MAX - 1) return fail(h, PT_ERR_ARG, "a spin's sum of |J| exceeds 127");
    const int kt = table_rows_for(kmax);
    if (kt <= h->kt) return PT_OK;
    Tables tb;
    const std::string why = build_tables(h->NT, kt, h->betas.data(), tb);
    if (!why.empty()) return fail(h, PT_ERR_ARG, why);
    uint32_t* d = nullptr;
    CK(dalloc(&d, tb.thr.size()), "cudaMalloc thr");
    cudaError_t e = cudaMemcpy(d, tb.thr.data(), 4 * tb.thr.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);     // no launch still reads the old table
    if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_fail(h, e, "upload thr");
    }
    const int old_kt = h->kt;
    uint32_t* old = h->d_thr;
    h->d_thr = d;
    h->kt = kt;
    for (Group* g : {&h->main, &h->cand}) {
        for (InstDesc& x : g->desc) { x.thr = d; x.kt = kt; }
        if (g->n_inst == 0) continue;
        int rc = upload_desc(h, *g);
        if (!rc) rc = group_schedule(h, *g);
        if (rc) {                                   // keep the old, still valid table
            h->d_thr = old;
            h->kt = old_kt;
            for (Group* g2 : {&h->main, &h->cand}) {
                for (InstDesc& x : g2->desc) { x.thr = old; x.kt = old_kt; }
                if (g2->n_inst) { upload_desc(h, *g2); group_schedule(h, *g2); }
            }
            cudaFree(d);
            return rc;
        }
    }
    cudaFree(old);
    h->tb = std::move(tb);
    return PT_OK;
}

}  // namespace

void ptg::set_global_error(const char* msg)
{
    std::lock_guard<std::mutex> g(g_err_mu);
    g_create_err = msg;
}

// ==========================================================================
// C ABI
// ==========================================================================
extern "C" {

const char* pt_last_error(const pt_handle* h)
{
    if (h) return h->err.c_str();
    std::lock_guard<std::mutex> g(g_err_mu);
    return g_create_err.c_str();
}

int pt_create(pt_handle** out, int32_t L, const int8_t* J, int32_t n_edges, const double* betas,
              int32_t n_temps, int32_t n_runs, uint32_t seed, uint32_t uid, void* stream)
{
    pt_handle* h = nullptr;
    if (!out || !J || !betas) return fail(nullptr, PT_ERR_ARG, "NULL argument");
    *out = nullptr;
    if (L < 1 || L > MAX_L) return fail(nullptr, PT_ERR_ARG, "chimera_L must be in [1, 16]");
    if (n_edges != n_edges_of(L)) return fail(nullptr, PT_ERR_ARG, "n_edges != 16 L^2 + 8 L (L-1)");
    if (n_temps < 1 || n_temps > MAX_TEMPS) return fail(nullptr, PT_ERR_ARG, "n_temps must be in [1, 64]");
    if (n_runs < 1 || n_runs > 1024) return fail(nullptr, PT_ERR_ARG, "n_runs must be in [1, 1024]");
    for (int e = 0; e < n_edges; ++e)
        if (J[e] < -J_ABS_MAX) return fail(nullptr, PT_ERR_ARG, "coupler outside [-127, 127]");
    const int kmax = coupler_kmax(L, J);
    if (kmax > KT_MAX - 1) return fail(nullptr, PT_ERR_ARG, "a spin's sum of |J| exceeds 127");
    for (int t = 0; t < n_temps; ++t) {
        if (!(betas[t] > 0.0) || !std::isfinite(betas[t])) return fail(nullptr, PT_ERR_ARG, "beta must be finite and > 0");
        if (t > 0 && !(betas[t] < betas[t - 1])) return fail(nullptr, PT_ERR_ARG, "betas must be strictly descending");
    }
    h = new (std::nothrow) pt_handle();
    if (!h) return fail(nullptr, PT_ERR_OOM, "host allocation failed");
    h->L = L; h->NT = n_temps; h->R = n_runs; h->N = 8 * L * L; h->n_edges = n_edges;
    h->seed = seed; h->uid = uid;
    h->J.assign(J, J + n_edges);
    h->betas.assign(betas, betas + n_temps);
    h->kt = table_rows_for(kmax);
    std::string why = build_tables(n_temps, h->kt, betas, h->tb);
    if (!why.empty()) { delete h; return fail(nullptr, PT_ERR_ARG, why); }
    int rc = PT_OK;
    auto bail = [&](int code) { std::string m = h->err; pt_destroy(h); return fail(nullptr, code, m); };
    if (stream) h->stream = (cudaStream_t)stream;
    else {
        cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { cuda_fail(h, e, "cudaStreamCreate"); return bail(PT_ERR_CUDA); }
        h->own_stream = true;
    }
#define CKC(call, what)                                                       \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) { int c_ = cuda_fail(h, e_, what); return bail(c_); } \
    } while (0)
    const int64_t xt = (int64_t)h->tb.xthr.size();
    std::vector<int32_t> xoff32(h->tb.xoff.begin(), h->tb.xoff.end());
    std::vector<int16_t> nbr((size_t)L * L * 4);
    build_neighbours(L, nbr.data());
    CKC(dalloc(&h->d_thr, h->tb.thr.size()), "cudaMalloc thr");
    CKC(dalloc(&h->d_xoff, xoff32.size()), "cudaMalloc xoff");
    CKC(dalloc(&h->d_xthr, (size_t)xt), "cudaMalloc xthr");
    CKC(dalloc(&h->d_xhint, h->tb.xhint.size()), "cudaMalloc xhint");
    CKC(dalloc(&h->d_nbr, nbr.size()), "cudaMalloc nbr");
    CKC(cudaMemcpy(h->d_thr, h->tb.thr.data(), 4 * h->tb.thr.size(), cudaMemcpyHostToDevice), "upload thr");
    CKC(cudaMemcpy(h->d_xoff, xoff32.data(), 4 * xoff32.size(), cudaMemcpyHostToDevice), "upload xoff");
    if (xt) CKC(cudaMemcpy(h->d_xthr, h->tb.xthr.data(), 4 * (size_t)xt, cudaMemcpyHostToDevice), "upload xthr");
    CKC(cudaMemcpy(h->d_xhint, h->tb.xhint.data(), 4 * h->tb.xhint.size(), cudaMemcpyHostToDevice), "upload xhint");
    CKC(cudaMemcpy(h->d_nbr, nbr.data(), 2 * nbr.size(), cudaMemcpyHostToDevice), "upload nbr");
    default_schedule(L, n_temps, n_runs, h->sp, h->ipc, h->kt);
    if ((rc = group_alloc(h, h->main, 1))) return bail(rc);
    if ((rc = group_schedule(h, h->main))) return bail(rc);
    if ((rc = upload_couplers(h, h->main, 0, h->J.data()))) return bail(rc);
    if ((rc = upload_desc(h, h->main))) return bail(rc);
    if ((rc = group_reset(h, h->main, true))) return bail(rc);
    CKC(cudaStreamSynchronize(h->stream), "sync after create");
#undef CKC
    *out = h;
    return PT_OK;
}

int pt_create_graph(pt_handle** out, const pt_graph* g, const int8_t* J, const double* betas, int32_t n_temps,
                    int32_t n_runs, uint32_t seed, uint32_t uid, void* stream)
{
    if (!out || !g || !J) return fail(nullptr, PT_ERR_ARG, "NULL argument");
    *out = nullptr;
    const int L = g->chimera_L;
    if (L < 1 || L > MAX_L) return fail(nullptr, PT_ERR_ARG, "chimera_L must be in [1, 16]");
    if (!g->ei && !g->ej) return pt_create(out, L, J, g->n_edges, betas, n_temps, n_runs, seed, uid, stream);
    if (!g->ei || !g->ej) return fail(nullptr, PT_ERR_ARG, "ei and ej must both be given or both be NULL");
    const int N = 8 * L * L, E = n_edges_of(L);
    if (g->n != N) return fail(nullptr, PT_ERR_ARG, "n must be 8 L^2 (the spins of C_L)");
    if (g->n_edges < 0 || g->n_edges > E) return fail(nullptr, PT_ERR_ARG, "more couplers than C_L has");
    // library index of the Chimera coupler (a, b), or -1 when (a, b) is not one
    auto edge_of = [L, N](int a, int b) -> int {
        if (a < 0 || b < 0 || a >= N || b >= N || a == b) return -1;
        int ca = a >> 3, cb = b >> 3, ua = (a >> 2) & 1, ub = (b >> 2) & 1, ka = a & 3, kb = b & 3;
        if (ca == cb) {
            if (ua == ub) return -1;
            const int kv = ua == 0 ? ka : kb, kh = ua == 0 ? kb : ka;
            return intra_edge(L, ca, kv, kh);
        }
        if (ua != ub || ka != kb) return -1;
        if (ca > cb) { std::swap(ca, cb); }
        const int r = ca / L, c = ca % L, r2 = cb / L, c2 = cb % L;
        if (ua == 0 && c == c2 && r2 == r + 1) return vert_edge(L, r, c, ka);
        if (ua == 1 && r == r2 && c2 == c + 1) return horiz_edge(L, r, c, ka);
        return -1;
    };
    std::vector<int8_t> full((size_t)E, 0);
    std::vector<char> seen((size_t)E, 0);
    for (int e = 0; e < g->n_edges; ++e) {
        const int x = edge_of(g->ei[e], g->ej[e]);
        if (x < 0) return fail(nullptr, PT_ERR_ARG, "coupler " + std::to_string(e) + " is not an edge of C_L");
        if (seen[(size_t)x]) return fail(nullptr, PT_ERR_ARG, "coupler " + std::to_string(e) + " is listed twice");
        seen[(size_t)x] = 1;
        full[(size_t)x] = J[e];
    }
    return pt_create(out, L, full.data(), E, betas, n_temps, n_runs, seed, uid, stream);
}

void pt_destroy(pt_handle* h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_group(h->main);
    free_group(h->cand);
    cudaFree(h->d_thr); cudaFree(h->d_xoff); cudaFree(h->d_xthr); cudaFree(h->d_xhint); cudaFree(h->d_nbr);
    for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
    if (h->eb0) cudaEventDestroy(h->eb0);
    if (h->eb1) cudaEventDestroy(h->eb1);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

int pt_reset(pt_handle* h, uint32_t uid)
{
    if (!h) return PT_ERR_ARG;
    h->uid = uid;
    h->main.desc[0].uid = uid;
    int rc;
    if ((rc = upload_desc(h, h->main))) return rc;
    if ((rc = group_reset(h, h->main, true))) return rc;
    CK(cudaStreamSynchronize(h->stream), "sync reset");
    return PT_OK;
}

int pt_set_spins(pt_handle* h, const int8_t* spins)
{
    if (!h || !spins) return fail(h, PT_ERR_ARG, "NULL argument");
    const size_t n = (size_t)h->R * h->NT * h->N;
    for (size_t i = 0; i < n; ++i)
        if (spins[i] != 1 && spins[i] != -1) return fail(h, PT_ERR_ARG, "spins must be +-1");
    CK(cudaMemcpyAsync(h->main.spins, spins, n, cudaMemcpyHostToDevice, h->stream), "upload spins");
    CK(launch_init(h->main.d_desc, h->main.d_items, h->R, false, h->stream), "init kernel");
    CK(launch_energy(h->main.d_desc, h->main.d_items, h->R, (int32_t)h->main.sweep, h->stream), "energy kernel");
    h->launches += 2;
    int rc = walk_clear(h, h->main);
    if (rc) return rc;
    CK(cudaStreamSynchronize(h->stream), "sync set_spins");
    return PT_OK;
}

int pt_sweep(pt_handle* h, int32_t n_sweeps, int32_t exchange_every)
{
    if (!h) return PT_ERR_ARG;
    if (n_sweeps < 0 || n_sweeps > (1 << 24) || exchange_every < 0)
        return fail(h, PT_ERR_ARG, "n_sweeps must be in [0, 2^24], exchange_every >= 0");
    if (h->main.sweep + (uint64_t)n_sweeps > 0x7FFFFFFFull) return fail(h, PT_ERR_STATE, "sweep counter would exceed 2^31-1");
    int rc = group_sweeps(h, h->main, n_sweeps, exchange_every);
    if (rc) return rc;
    CK(cudaStreamSynchronize(h->stream), "sync sweep");
    return collect_timing(h);
}

int pt_exchange(pt_handle* h)
{
    if (!h) return PT_ERR_ARG;
    Group& g = h->main;
    CK(launch_sweeps(g.d_desc, g.d_bundles, (int)g.bundles.size(), (int)g.bundles.size(), g.block,
                     g.smem, (uint32_t)g.sweep, 0, 0, 1, nullptr, h->stream, h->team > 0, g.walk, g.L),
       "exchange kernel");
    ++h->launches;
    if (g.walk && g.NT > 1) g.walk_passes += 1;
    CK(cudaStreamSynchronize(h->stream), "sync exchange");
    return PT_OK;
}

int pt_get_state(pt_handle* h, int8_t* spins, int32_t* E, uint8_t* perm, int32_t* best, int32_t* first,
                 uint64_t* macc, uint64_t* xacc, uint64_t* sweep)
{
    if (!h) return PT_ERR_ARG;
    Group& g = h->main;
    const size_t reps = (size_t)h->R * h->NT, N = h->N;
    std::vector<uint8_t> pm(reps);
    CK(cudaMemcpyAsync(pm.data(), g.perm, reps, cudaMemcpyDeviceToHost, h->stream), "download perm");
    std::vector<int8_t> sp;
    if (spins) {
        sp.resize(reps * N);
        CK(cudaMemcpyAsync(sp.data(), g.spins, reps * N, cudaMemcpyDeviceToHost, h->stream), "download spins");
    }
    if (E) CK(cudaMemcpyAsync(E, g.E, 4 * reps, cudaMemcpyDeviceToHost, h->stream), "download E");
    if (best) CK(cudaMemcpyAsync(best, g.best, 4 * (size_t)h->R, cudaMemcpyDeviceToHost, h->stream), "download best");
    if (first) CK(cudaMemcpyAsync(first, g.first, 4 * (size_t)h->R, cudaMemcpyDeviceToHost, h->stream), "download first");
    if (macc) CK(cudaMemcpyAsync(macc, g.macc, 8 * reps, cudaMemcpyDeviceToHost, h->stream), "download macc");
    if (xacc && h->NT > 1)
        CK(cudaMemcpyAsync(xacc, g.xacc, 8 * (size_t)h->R * (h->NT - 1), cudaMemcpyDeviceToHost, h->stream), "download xacc");
    CK(cudaStreamSynchronize(h->stream), "sync get_state");
    if (perm) std::memcpy(perm, pm.data(), reps);
    if (spins)   // slot order: slot t holds buffer perm[t]
        for (int r = 0; r < h->R; ++r)
            for (int t = 0; t < h->NT; ++t)
                std::memcpy(spins + ((size_t)r * h->NT + t) * N,
                            sp.data() + ((size_t)r * h->NT + pm[(size_t)r * h->NT + t]) * N, N);
    if (sweep) *sweep = g.sweep;
    return PT_OK;
}

int pt_tts(pt_handle* h, int32_t E_target, int32_t horizon, int32_t* tts, int32_t* n_hit, int32_t* target_used)
{
    if (!h || !tts) return fail(h, PT_ERR_ARG, "NULL argument");
    if (horizon < 0 || horizon == INT32_MAX) return fail(h, PT_ERR_ARG, "horizon must be in [0, 2^31-2]");
    std::vector<int32_t> out;
    int rc = group_tts(h, h->main, E_target, horizon, out);
    if (rc) return rc;
    *tts = out[0];
    if (n_hit) *n_hit = out[1];
    if (target_used) *target_used = out[2];
    return PT_OK;
}

int pt_tts_eval(pt_handle* h, uint32_t uid, int32_t S, int32_t pass_mult, int32_t xevery,
                int32_t* tts, int32_t* n_hit, int32_t* target)
{
    if (!h || !tts) return fail(h, PT_ERR_ARG, "NULL argument");
    if (S < 1 || pass_mult < 1 || xevery < 0 || (int64_t)S * pass_mult > (1 << 30))
        return fail(h, PT_ERR_ARG, "need S >= 1, pass_mult >= 1, S * pass_mult <= 2^30");
    h->uid = uid;
    h->main.desc[0].uid = uid;
    std::vector<int32_t> out;
    int rc = group_eval(h, h->main, S, pass_mult, xevery, out);
    if (rc) return rc;
    *tts = out[0];
    if (n_hit) *n_hit = out[1];
    if (target) *target = out[2];
    return PT_OK;
}

int pt_tts_eval_doubling(pt_handle* h, uint32_t uid, int32_t S0, int32_t Smax, int32_t xevery, int32_t* tts,
                         int32_t* n_hit, int32_t* target, int32_t* level)
{
    if (!h || !tts) return fail(h, PT_ERR_ARG, "NULL argument");
    if (!doubling_ok(S0, Smax, 1) || xevery < 0)
        return fail(h, PT_ERR_ARG, "need S0 >= 1, Smax = S0 * 2^k <= 2^30, exchange_every >= 0");
    h->uid = uid;
    h->main.desc[0].uid = uid;
    std::vector<int32_t> out, levels;
    int rc = group_eval_doubling(h, h->main, S0, Smax, xevery, out, levels);
    if (rc) return rc;
    *tts = out[0];
    if (n_hit) *n_hit = out[1];
    if (target) *target = out[2];
    if (level) *level = levels[0];
    return PT_OK;
}

int pt_tts_eval_many(pt_handle* h, int32_t k, const int8_t* J, const uint32_t* uids, int32_t S, int32_t pass_mult,
                     int32_t max_sweeps, int32_t xevery, int32_t* tts, int32_t* n_hit, int32_t* target,
                     int32_t* level)
{
    if (!h || !J || !uids || !tts) return fail(h, PT_ERR_ARG, "NULL argument");
    if (k < 1 || k > 256) return fail(h, PT_ERR_ARG, "need 1 <= k <= 256");
    if (S < 1 || pass_mult < 1 || xevery < 0 || (int64_t)S * pass_mult > (1 << 30))
        return fail(h, PT_ERR_ARG, "need S >= 1, pass_mult >= 1, S * pass_mult <= 2^30");
    if (max_sweeps != 0 && !doubling_ok(S, max_sweeps, pass_mult))
        return fail(h, PT_ERR_ARG, "max_sweeps must be S * 2^k <= 2^30 with pass_mult 1");
    for (size_t i = 0; i < (size_t)k * h->n_edges; ++i)
        if (J[i] < -J_ABS_MAX) return fail(h, PT_ERR_ARG, "coupler outside [-127, 127]");
    const pt_rule keep = h->rule;
    h->rule.S = S;
    h->rule.pass_mult = pass_mult;
    h->rule.max_sweeps = max_sweeps;
    h->rule.exchange_every = xevery;
    std::vector<int32_t> res;
    int rc = eval_candidates(h, k, J, uids, res);
    const std::vector<int32_t> lv = h->last_levels;
    h->rule = keep;
    if (rc) return rc;
    for (int j = 0; j < k; ++j) {
        tts[j] = res[(size_t)j * 3];
        if (n_hit) n_hit[j] = res[(size_t)j * 3 + 1];
        if (target) target[j] = res[(size_t)j * 3 + 2];
        if (level) level[j] = max_sweeps > 0 ? lv[(size_t)j] : S * pass_mult;
    }
    return PT_OK;
}

int pt_set_coupler(pt_handle* h, int32_t edge, int8_t value)
{
    if (!h) return PT_ERR_ARG;
    if (edge < 0 || edge >= h->n_edges || value < -J_ABS_MAX)
        return fail(h, PT_ERR_ARG, "edge out of range or |value| > 127");
    const int8_t prev = h->J[edge];
    h->spec_cache.valid = false;
    h->lao_cache.valid = false;
    h->J[edge] = value;
    if (int rc0 = ensure_table_rows(h, coupler_kmax(h->L, h->J.data()))) {
        h->J[edge] = prev;
        return rc0;
    }
    int rc = upload_couplers(h, h->main, 0, h->J.data());
    if (rc) return rc;
    CK(launch_energy(h->main.d_desc, h->main.d_items, h->R, (int32_t)h->main.sweep, h->stream), "energy kernel");
    ++h->launches;
    CK(cudaStreamSynchronize(h->stream), "sync set_coupler");
    return PT_OK;
}

int pt_get_couplers(pt_handle* h, int8_t* J)
{
    if (!h || !J) return fail(h, PT_ERR_ARG, "NULL argument");
    std::memcpy(J, h->J.data(), h->J.size());
    return PT_OK;
}

int pt_get_tables(const pt_handle* h, uint32_t* thr, int64_t* xoff, uint32_t* xthr, int64_t cap, int64_t* len)
{
    if (!h) return PT_ERR_ARG;
    const int64_t n = (int64_t)h->tb.xthr.size();
    if (len) *len = n;
    if (thr) std::memcpy(thr, h->tb.thr.data(), 4 * h->tb.thr.size());
    if (xoff) std::memcpy(xoff, h->tb.xoff.data(), 8 * h->tb.xoff.size());
    if (xthr) {
        if (cap < n) return PT_ERR_ARG;
        std::memcpy(xthr, h->tb.xthr.data(), 4 * (size_t)n);
    }
    return PT_OK;
}

int pt_debug_enabled(void) { return debug_build() ? 1 : 0; }

int pt_debug_status(uint32_t* code)
{
    if (!code) return PT_ERR_ARG;
    *code = debug_take();
    return PT_OK;
}

int pt_get_table_rows(const pt_handle* h, int32_t* rows)
{
    if (!h || !rows) return PT_ERR_ARG;
    *rows = h->kt;
    return PT_OK;
}

int engineer_begin(pt_handle* h, const pt_rule* rule, uint32_t base_uid, int32_t* tts0)
{
    if (!h || !rule) return fail(h, PT_ERR_ARG, "NULL argument");
    if (rule->S < 1 || rule->pass_mult < 1 || rule->exchange_every < 0 ||
        (rule->direction != 1 && rule->direction != -1) || (int64_t)rule->S * rule->pass_mult > (1 << 30))
        return fail(h, PT_ERR_ARG, "invalid pt_rule");
    if (rule->max_sweeps != 0 && !doubling_ok(rule->S, rule->max_sweeps, rule->pass_mult))
        return fail(h, PT_ERR_ARG, "max_sweeps must be S * 2^k <= 2^30 with pass_mult 1");
    h->rule = *rule;
    h->base_uid = base_uid;
    h->spec_cache.valid = false;
    h->lao_cache.valid = false;
    int32_t t, nh;
    int rc = rule->max_sweeps > 0
                 ? pt_tts_eval_doubling(h, base_uid, rule->S, rule->max_sweeps, rule->exchange_every, &t, &nh,
                                        nullptr, nullptr)
                 : pt_tts_eval(h, base_uid, rule->S, rule->pass_mult, rule->exchange_every, &t, &nh, nullptr);
    if (rc) return rc;
    h->tts_cur = t;
    h->hits_cur = nh;
    h->eng = true;
    h->lao = false;
    if (tts0) *tts0 = t;
    return PT_OK;
}

int engineer_run(pt_handle* h, uint32_t step0, int32_t n_steps, int32_t spec, pt_step_result* out)
{
    if (!h) return PT_ERR_ARG;
    if (!h->eng) return fail(h, PT_ERR_STATE, "engineer_begin not called");
    if (n_steps < 0 || spec < 1 || spec > 16) return fail(h, PT_ERR_ARG, "need n_steps >= 0, speculation in [1, 16]");
    int rc = ensure_candidates(h, spec);
    if (rc) return rc;
    std::vector<int8_t> Jc((size_t)spec * h->n_edges);
    std::vector<int32_t> e(spec), v(spec), res, lv;
    std::vector<uint32_t> cu(spec), ua(spec);
    pt_handle::SpecCache& c = h->spec_cache;
    h->lao_cache.valid = false;                // LAO's kept evaluations assume the LAO state
    int32_t done = 0;
    bool changed = false;
    while (done < n_steps) {
        const uint32_t s0 = step0 + (uint32_t)done;
        const int n = h->adapt ? h->n_cur : h->R;
        // candidates of steps s0, s0+1, ...: evaluated by the previous call past its end, if nothing
        // their evaluation depends on has changed since; otherwise a full batch of spec is evaluated
        // now, so that the GPU holds spec candidates' runs even when fewer steps remain in this call
        int k;
        if (c.valid && c.step == s0 && c.n_runs == n && c.base_uid == h->base_uid && c.rule.S == h->rule.S &&
            c.rule.pass_mult == h->rule.pass_mult && c.rule.exchange_every == h->rule.exchange_every &&
            c.rule.max_sweeps == h->rule.max_sweeps && c.J == h->J) {
            k = (int)c.e.size();
            e = c.e; v = c.v; cu = c.cu; ua = c.ua; res = c.res; lv = c.level;
        } else {
            k = spec;
            e.resize(k); v.resize(k); cu.resize(k); ua.resize(k);
            for (int j = 0; j < k; ++j) {
                engineer_draw(h, h->J.data(), s0 + (uint32_t)j, 0u, e[j], v[j], cu[j], ua[j]);
                int8_t* Jj = Jc.data() + (size_t)j * h->n_edges;
                std::memcpy(Jj, h->J.data(), h->n_edges);
                Jj[e[j]] = (int8_t)v[j];
            }
            // every candidate of the batch uses the runs of the step it stands for
            rc = eval_candidates(h, k, Jc.data(), cu.data(), res, PT_TARGET_BEST, nullptr, n);
            if (rc) return rc;
            lv.assign(h->last_levels.begin(), h->last_levels.begin() + k);
        }
        c.valid = false;
        pt_rule rule = h->rule;
        if (h->adapt && h->beta_per_run > 0.0) rule.beta_rao = h->beta_per_run * (double)n;
        // decisions in step order; the batch is cut after a candidate that is kept or that halves the runs
        const int kuse = std::min<int>(k, n_steps - done);
        int used = kuse;
        bool stop = false;
        for (int j = 0; j < kuse && !stop; ++j) {
            const int32_t tn = res[(size_t)j * 3];
            const int32_t level = lv[(size_t)j];
            const bool acc = engineer_accept(rule, h->tts_cur, tn, ua[j]);
            if (out) {
                pt_step_result& o = out[done + j];
                o.edge = e[j]; o.old_value = h->J[e[j]]; o.new_value = v[j];
                o.tts_old = h->tts_cur; o.tts_new = tn; o.accepted = acc ? 1 : 0; o.cand_uid = cu[j];
                o.n_runs = n; o.level = level;
            }
            if (acc) {
                h->J[e[j]] = (int8_t)v[j];
                h->tts_cur = tn;
                h->hits_cur = res[(size_t)j * 3 + 1];
                changed = true;
                stop = true;
            }
            if (h->adapt && (int64_t)n * level > h->cost_max && n > h->n_min) {
                h->n_cur = std::max(h->n_min, n / 2);
                stop = true;
            }
            if (stop) used = j + 1;
        }
        if (!stop && kuse < k) {               // steps past this call's end: kept for the next call
            c.valid = true;
            c.step = s0 + (uint32_t)kuse;
            c.n_runs = n;
            c.base_uid = h->base_uid;
            c.rule = h->rule;
            c.J = h->J;
            c.e.assign(e.begin() + kuse, e.begin() + k);
            c.v.assign(v.begin() + kuse, v.begin() + k);
            c.cu.assign(cu.begin() + kuse, cu.begin() + k);
            c.ua.assign(ua.begin() + kuse, ua.begin() + k);
            c.res.assign(res.begin() + (size_t)kuse * 3, res.begin() + (size_t)k * 3);
            c.level.assign(lv.begin() + kuse, lv.begin() + k);
        }
        done += used;
    }
    if (changed) {
        rc = upload_couplers(h, h->main, 0, h->J.data());
        if (rc) return rc;
    }
    return PT_OK;
}

int engineer_step(pt_handle* h, uint32_t step, pt_step_result* out)
{
    return engineer_run(h, step, 1, 1, out);
}

int lao_plant(int32_t chimera_L, uint32_t seed, uint32_t uid, int32_t n_loops, int32_t w_max, int8_t* planted,
              int32_t* loops, int8_t* J, int32_t* E_gs)
{
    if (!planted || !loops || !J || !E_gs) return fail(nullptr, PT_ERR_ARG, "NULL argument");
    if (chimera_L < 1 || chimera_L > MAX_L || n_loops < 1 || w_max < 1 || w_max > J_ABS_MAX)
        return fail(nullptr, PT_ERR_ARG, "need 1 <= L <= 16, n_loops >= 1, 1 <= w_max <= 127");
    const LaoGraph g(chimera_L);
    for (int i = 0; i < g.N; ++i)
        planted[i] = (lao_word(seed, uid, 0u, 0xFFFFFFF0u, (uint32_t)(i >> 2), i & 3) >> 31) ? -1 : 1;
    std::memset(J, 0, (size_t)g.E);
    for (int m = 0; m < n_loops; ++m) {
        int32_t* rec = loops + (size_t)m * PT_LOOP_WORDS;
        if (!lao_draw_loop(g, planted, J, seed, uid, 0u, (uint32_t)m, (int)w_max, rec))
            return fail(nullptr, PT_ERR_STATE, "no admissible loop (the couplers would leave the engine's bounds)");
        loop_apply(g, planted, rec, J, 1);
    }
    *E_gs = loops_gs(loops, n_loops);
    return PT_OK;
}

int lao_begin(pt_handle* h, const pt_rule* rule, uint32_t uid, int32_t n_loops, int32_t w_max, int32_t* tts0)
{
    if (!h || !rule) return fail(h, PT_ERR_ARG, "NULL argument");
    if (rule->S < 1 || rule->exchange_every < 0 || (rule->direction != 1 && rule->direction != -1) ||
        rule->S > (1 << 30))
        return fail(h, PT_ERR_ARG, "invalid pt_rule");
    std::vector<int8_t> planted(h->N), J(h->n_edges);
    std::vector<int32_t> loops((size_t)std::max(n_loops, 1) * PT_LOOP_WORDS);
    int32_t eg = 0;
    if (lao_plant(h->L, h->seed, uid, n_loops, w_max, planted.data(), loops.data(), J.data(), &eg) != PT_OK)
        return fail(h, PT_ERR_ARG, pt_last_error(nullptr));
    h->spec_cache.valid = false;
    h->lao_cache.valid = false;
    h->rule = *rule;
    h->rule.pass_mult = 1;                   // the target is known: no longer pass
    h->rule.max_sweeps = 0;                  // one pass of S sweeps against E_GS
    h->planted = planted;
    h->loops = loops;
    h->J = J;
    h->E_gs = eg;
    h->lao_uid = uid;
    h->lao_w_max = w_max;
    int rc = upload_couplers(h, h->main, 0, h->J.data());
    if (rc) return rc;
    const uint32_t u0 = lao_word(h->seed, uid, 0u, 0xFFFFFFFEu, 0u, 2);
    std::vector<int32_t> res;
    if ((rc = eval_candidates(h, 1, h->J.data(), &u0, res, h->E_gs))) return rc;
    h->tts_cur = res[0];
    h->hits_cur = res[1];
    h->lao = true;
    h->eng = false;
    if (tts0) *tts0 = h->tts_cur;
    return PT_OK;
}

int lao_run(pt_handle* h, uint32_t step0, int32_t n_steps, int32_t spec, pt_lao_result* out)
{
    if (!h) return PT_ERR_ARG;
    h->spec_cache.valid = false;           // the couplers change outside engineer_run
    if (!h->lao) return fail(h, PT_ERR_STATE, "lao_begin not called");
    if (step0 < 1 || n_steps < 0 || spec < 1 || spec > 16)
        return fail(h, PT_ERR_ARG, "need step0 >= 1, n_steps >= 0, speculation in [1, 16]");
    int rc = ensure_candidates(h, spec);
    if (rc) return rc;
    const LaoGraph g(h->L);
    const int M = (int)(h->loops.size() / PT_LOOP_WORDS);
    std::vector<int8_t> Jc((size_t)spec * h->n_edges);
    std::vector<int32_t> rem(spec), egs(spec), recs((size_t)spec * PT_LOOP_WORDS);
    std::vector<uint32_t> cu(spec), ua(spec);
    int32_t done = 0;
    bool changed = false;
    pt_handle::LaoCache& c = h->lao_cache;
    while (done < n_steps) {
        const uint32_t s0 = step0 + (uint32_t)done;
        // candidates drawn against the current instance: after the first accepted one the rest are stale
        // and redrawn (same results as one by one).  Evaluations the previous call made for steps past
        // its end are used if the instance, its loops and E_GS are unchanged; otherwise a full batch of
        // spec is evaluated, also when fewer steps remain in this call.
        int k;
        std::vector<int32_t> res;
        if (c.valid && c.step == s0 && c.rule.S == h->rule.S && c.rule.exchange_every == h->rule.exchange_every &&
            c.E_gs == h->E_gs && c.J == h->J && c.loops == h->loops) {
            k = (int)c.rem.size();
            Jc = c.Jc; rem = c.rem; egs = c.egs; recs = c.recs; res = c.res; cu = c.cu; ua = c.ua;
        } else {
            k = spec;
            Jc.resize((size_t)k * h->n_edges);
            rem.resize(k); egs.resize(k); recs.resize((size_t)k * PT_LOOP_WORDS); cu.resize(k); ua.resize(k);
            for (int j = 0; j < k; ++j) {
                const uint32_t t = s0 + (uint32_t)j;
                uint32_t ctl[3];
                for (int w = 0; w < 3; ++w) ctl[w] = lao_word(h->seed, h->lao_uid, t, 0xFFFFFFFEu, 0u, w);
                rem[j] = (int)mulhi(ctl[0], (uint32_t)M);
                ua[j] = ctl[1];
                cu[j] = ctl[2];
                const int32_t* old = h->loops.data() + (size_t)rem[j] * PT_LOOP_WORDS;
                int8_t* Jj = Jc.data() + (size_t)j * h->n_edges;
                int32_t* rec = recs.data() + (size_t)j * PT_LOOP_WORDS;
                std::memcpy(Jj, h->J.data(), h->n_edges);
                loop_apply(g, h->planted.data(), old, Jj, -1);
                if (!lao_draw_loop(g, h->planted.data(), Jj, h->seed, h->lao_uid, t, 0xFFFFFFFFu, h->lao_w_max, rec))
                    return fail(h, PT_ERR_STATE, "no admissible replacement loop");
                loop_apply(g, h->planted.data(), rec, Jj, 1);
                egs[j] = h->E_gs + old[1] * (old[0] - 2) - rec[1] * (rec[0] - 2);
            }
            // one batched evaluation, each candidate against its own ground-state energy
            if ((rc = eval_candidates(h, k, Jc.data(), cu.data(), res, PT_TARGET_BEST, egs.data()))) return rc;
        }
        c.valid = false;
        const int kuse = std::min<int>(k, n_steps - done);
        int used = kuse;
        bool kept = false;
        for (int j = 0; j < kuse; ++j) {
            const int32_t tn = res[(size_t)j * 3];
            const bool acc = engineer_accept(h->rule, h->tts_cur, tn, ua[j]);
            if (out) {
                pt_lao_result& o = out[done + j];
                o.removed = rem[j];
                std::memcpy(o.loop, recs.data() + (size_t)j * PT_LOOP_WORDS, sizeof(o.loop));
                o.E_gs_new = egs[j];
                o.tts_old = h->tts_cur;
                o.tts_new = tn;
                o.accepted = acc ? 1 : 0;
                o.cand_uid = cu[j];
            }
            if (acc) {
                std::memcpy(h->J.data(), Jc.data() + (size_t)j * h->n_edges, h->n_edges);
                std::memcpy(h->loops.data() + (size_t)rem[j] * PT_LOOP_WORDS, recs.data() + (size_t)j * PT_LOOP_WORDS,
                            sizeof(int32_t) * PT_LOOP_WORDS);
                h->E_gs = egs[j];
                h->tts_cur = tn;
                h->hits_cur = res[(size_t)j * 3 + 1];
                changed = true;
                kept = true;
                used = j + 1;
                break;
            }
        }
        if (!kept && kuse < k) {               // steps past this call's end: kept for the next call
            c.valid = true;
            c.step = s0 + (uint32_t)kuse;
            c.rule = h->rule;
            c.J = h->J;
            c.loops = h->loops;
            c.E_gs = h->E_gs;
            c.Jc.assign(Jc.begin() + (size_t)kuse * h->n_edges, Jc.begin() + (size_t)k * h->n_edges);
            c.rem.assign(rem.begin() + kuse, rem.begin() + k);
            c.egs.assign(egs.begin() + kuse, egs.begin() + k);
            c.recs.assign(recs.begin() + (size_t)kuse * PT_LOOP_WORDS, recs.begin() + (size_t)k * PT_LOOP_WORDS);
            c.res.assign(res.begin() + (size_t)kuse * 3, res.begin() + (size_t)k * 3);
            c.cu.assign(cu.begin() + kuse, cu.begin() + k);
            c.ua.assign(ua.begin() + kuse, ua.begin() + k);
        }
        done += used;
    }
    if (changed) {
        rc = upload_couplers(h, h->main, 0, h->J.data());
        if (rc) return rc;
    }
    return PT_OK;
}

int pt_overlaps(pt_handle* h, int32_t E_gs, int32_t* n_gs, int32_t* n_es, int32_t* E1, double* q_gs_gs,
                double* q_gs_es)
{
    if (!h) return PT_ERR_ARG;
    Group& g = h->main;
    const int R = h->R, NT = h->NT;
    std::vector<int32_t> E((size_t)R * NT);
    CK(cudaMemcpyAsync(E.data(), g.E, sizeof(int32_t) * E.size(), cudaMemcpyDeviceToHost, h->stream), "download E");
    CK(cudaStreamSynchronize(h->stream), "sync overlaps");
    // E1: the lowest replica energy above E_gs; per run at most one sample of
    // each level, its coldest replica at that energy
    int32_t e1 = INT32_MAX;
    for (int32_t x : E) if (x > E_gs && x < e1) e1 = x;
    std::vector<int32_t> run, slot;
    int ngs = 0;
    for (int pass = 0; pass < 2; ++pass) {
        const int32_t level = pass == 0 ? E_gs : e1;
        for (int r = 0; r < R; ++r)
            for (int t = 0; t < NT; ++t)
                if (E[(size_t)r * NT + t] == level) {
                    run.push_back(r);
                    slot.push_back(t);
                    break;
                }
        if (pass == 0) ngs = (int)run.size();
    }
    const int n = (int)run.size(), nes = n - ngs;
    std::vector<int32_t> dist((size_t)n * n);
    if (n > 0) {
        int32_t *d = nullptr, *dr = nullptr, *ds = nullptr;
        cudaError_t e = dalloc(&d, (size_t)n * n);
        if (e == cudaSuccess) e = dalloc(&dr, (size_t)n);
        if (e == cudaSuccess) e = dalloc(&ds, (size_t)n);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dr, run.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(ds, slot.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = launch_hamming(g.d_desc, n, dr, ds, d, h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dist.data(), d, sizeof(int32_t) * dist.size(), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        ++h->launches;
        cudaFree(d); cudaFree(dr); cudaFree(ds);
        if (e != cudaSuccess) return cuda_fail(h, e, "overlaps");
    }
    // |q| = |1 - 2 h / N| (global flip symmetry); lower medians of the integers |N - 2 h|
    auto lower_median = [](std::vector<int32_t>& v) -> int32_t {
        if (v.empty()) return -1;
        std::sort(v.begin(), v.end());
        return v[(v.size() + 1) / 2 - 1];
    };
    std::vector<int32_t> a, b;
    for (int i = 0; i < ngs; ++i)
        for (int j = i + 1; j < ngs; ++j) a.push_back(std::abs(h->N - 2 * dist[(size_t)i * n + j]));
    for (int i = 0; i < ngs; ++i)
        for (int j = ngs; j < n; ++j) b.push_back(std::abs(h->N - 2 * dist[(size_t)i * n + j]));
    const int32_t ma = lower_median(a), mb = lower_median(b);
    if (n_gs) *n_gs = ngs;
    if (n_es) *n_es = nes;
    if (E1) *E1 = e1;
    if (q_gs_gs) *q_gs_gs = ma < 0 ? -1.0 : (double)ma / h->N;
    if (q_gs_es) *q_gs_es = mb < 0 ? -1.0 : (double)mb / h->N;
    return PT_OK;
}

int lao_state(const pt_handle* h, int8_t* planted, int32_t* loops, int8_t* J, int32_t* E_gs, int32_t* tts)
{
    if (!h || !h->lao) return PT_ERR_STATE;
    if (planted) std::memcpy(planted, h->planted.data(), h->planted.size());
    if (loops) std::memcpy(loops, h->loops.data(), sizeof(int32_t) * h->loops.size());
    if (J) std::memcpy(J, h->J.data(), h->J.size());
    if (E_gs) *E_gs = h->E_gs;
    if (tts) *tts = h->tts_cur;
    return PT_OK;
}

int engineer_guided_step(pt_handle* h, sg_model* m, uint32_t step, int32_t n_prop, int32_t top,
                         pt_step_result* out, float* pred, int32_t* ranked)
{
    if (!h) return fail(h, PT_ERR_ARG, "NULL argument");
    h->spec_cache.valid = false;           // the couplers change outside engineer_run
    h->lao_cache.valid = false;
    if (!h->eng) return fail(h, PT_ERR_STATE, "engineer_begin not called");
    if (n_prop < 1 || n_prop > 1024 || top < 1 || top > 16 || top > n_prop)
        return fail(h, PT_ERR_ARG, "need 1 <= top <= min(n_prop, 16), n_prop <= 1024");
    if (m)
        for (int e = 0; e < h->n_edges; ++e)
            if (h->J[e] == 0) return fail(h, PT_ERR_STATE, "the surrogate needs couplers in {+-1, +-2, +-3}");
    std::vector<int8_t> Jp((size_t)n_prop * h->n_edges);
    std::vector<int32_t> e(n_prop), v(n_prop);
    std::vector<uint32_t> cu(n_prop), ua(n_prop);
    for (int j = 0; j < n_prop; ++j) {
        engineer_draw(h, h->J.data(), step, (uint32_t)j, e[j], v[j], cu[j], ua[j]);
        int8_t* Jj = Jp.data() + (size_t)j * h->n_edges;
        std::memcpy(Jj, h->J.data(), h->n_edges);
        Jj[e[j]] = (int8_t)v[j];
    }
    std::vector<float> y(n_prop, 0.f);       // without a model every proposal ties: draw order
    if (m && sg_forward(m, h->L, n_prop, Jp.data(), y.data()) != PT_OK)
        return fail(h, PT_ERR_CUDA, std::string("surrogate forward: ") + sg_last_error(m));
    std::vector<int> order(n_prop);
    for (int j = 0; j < n_prop; ++j) order[j] = j;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return y[a] > y[b]; });
    std::vector<int8_t> Jc((size_t)top * h->n_edges);
    std::vector<uint32_t> uid(top);
    for (int r = 0; r < top; ++r) {
        std::memcpy(Jc.data() + (size_t)r * h->n_edges, Jp.data() + (size_t)order[r] * h->n_edges, h->n_edges);
        uid[r] = cu[order[r]];
    }
    std::vector<int32_t> res;
    int rc = eval_candidates(h, top, Jc.data(), uid.data(), res);
    if (rc) return rc;
    int best = 0;   // largest TTS in the direction of the rule; ties keep the better-ranked one
    for (int r = 1; r < top; ++r)
        if ((int64_t)h->rule.direction * ((int64_t)res[(size_t)r * 3] - res[(size_t)best * 3]) > 0) best = r;
    const int jb = order[best];
    const bool acc = engineer_accept(h->rule, h->tts_cur, res[(size_t)best * 3], ua[jb]);
    for (int r = 0; r < top; ++r) {
        const int j = order[r];
        if (out) {
            pt_step_result& o = out[r];
            o.edge = e[j]; o.old_value = h->J[e[j]]; o.new_value = v[j];
            o.tts_old = h->tts_cur; o.tts_new = res[(size_t)r * 3];
            o.accepted = (acc && r == best) ? 1 : 0; o.cand_uid = cu[j];
            o.n_runs = h->R; o.level = h->last_levels[(size_t)r];
        }
        if (ranked) ranked[r] = j;
    }
    if (pred) std::memcpy(pred, y.data(), sizeof(float) * n_prop);
    if (acc) {
        h->J[e[jb]] = (int8_t)v[jb];
        h->tts_cur = res[(size_t)best * 3];
        h->hits_cur = res[(size_t)best * 3 + 1];
        rc = upload_couplers(h, h->main, 0, h->J.data());
        if (rc) return rc;
    }
    return PT_OK;
}

int engineer_current_tts(const pt_handle* h, int32_t* tts)
{
    if (!h || !tts || !h->eng) return PT_ERR_STATE;
    *tts = h->tts_cur;
    return PT_OK;
}

int engineer_set_adaptive(pt_handle* h, int32_t n0, int32_t n_min, int64_t cost_max, double beta_per_run)
{
    if (!h) return PT_ERR_ARG;
    if (n0 == 0) {
        h->spec_cache.valid = false;
    h->lao_cache.valid = false;
        h->adapt = false;
        return PT_OK;
    }
    if (n_min < 1 || n0 < n_min || n0 > h->R || cost_max < 1 || !(beta_per_run >= 0.0) || !std::isfinite(beta_per_run))
        return fail(h, PT_ERR_ARG, "need 1 <= n_min <= n0 <= n_runs, cost_max >= 1, beta_per_run >= 0");
    h->spec_cache.valid = false;
    h->lao_cache.valid = false;
    h->adapt = true;
    h->n_cur = n0;
    h->n_min = n_min;
    h->cost_max = cost_max;
    h->beta_per_run = beta_per_run;
    return PT_OK;
}

int engineer_adaptive_runs(const pt_handle* h, int32_t* n)
{
    if (!h || !n) return PT_ERR_ARG;
    *n = h->adapt ? h->n_cur : h->R;
    return PT_OK;
}

int engineer_current_state(const pt_handle* h, int32_t* tts, int32_t* n_hit)
{
    if (!h || !(h->eng || h->lao)) return PT_ERR_STATE;
    if (tts) *tts = h->tts_cur;
    if (n_hit) *n_hit = h->hits_cur;
    return PT_OK;
}

int pt_checkpoint(pt_handle* h, void* buf, size_t* len)
{
    if (!h || !len) return fail(h, PT_ERR_ARG, "NULL argument");
    const size_t reps = (size_t)h->R * h->NT, npair = (size_t)h->R * (h->NT > 1 ? h->NT - 1 : 1);
    const size_t need = 64 + (size_t)h->n_edges + reps * h->N + 4 * reps + reps + 8 * (size_t)h->R +
                        8 * reps + 8 * npair;
    if (!buf) { *len = need; return PT_OK; }
    if (*len < need) return fail(h, PT_ERR_ARG, "checkpoint buffer too small");
    Group& g = h->main;
    uint8_t* p = static_cast<uint8_t*>(buf);
    int64_t hdr[8] = {0x5054434bLL, h->L, h->NT, h->R, (int64_t)g.sweep, (int64_t)h->uid, (int64_t)h->seed, 0};
    std::memcpy(p, hdr, 64); p += 64;
    std::memcpy(p, h->J.data(), h->n_edges); p += h->n_edges;
    CK(cudaMemcpyAsync(p, g.spins, reps * h->N, cudaMemcpyDeviceToHost, h->stream), "ckpt spins"); p += reps * h->N;
    CK(cudaMemcpyAsync(p, g.E, 4 * reps, cudaMemcpyDeviceToHost, h->stream), "ckpt E"); p += 4 * reps;
    CK(cudaMemcpyAsync(p, g.perm, reps, cudaMemcpyDeviceToHost, h->stream), "ckpt perm"); p += reps;
    CK(cudaMemcpyAsync(p, g.best, 4 * (size_t)h->R, cudaMemcpyDeviceToHost, h->stream), "ckpt best"); p += 4 * (size_t)h->R;
    CK(cudaMemcpyAsync(p, g.first, 4 * (size_t)h->R, cudaMemcpyDeviceToHost, h->stream), "ckpt first"); p += 4 * (size_t)h->R;
    CK(cudaMemcpyAsync(p, g.macc, 8 * reps, cudaMemcpyDeviceToHost, h->stream), "ckpt macc"); p += 8 * reps;
    CK(cudaMemcpyAsync(p, g.xacc, 8 * npair, cudaMemcpyDeviceToHost, h->stream), "ckpt xacc");
    CK(cudaStreamSynchronize(h->stream), "sync checkpoint");
    *len = need;
    return PT_OK;
}

int pt_restore(pt_handle* h, const void* buf, size_t len)
{
    if (!h || !buf) return fail(h, PT_ERR_ARG, "NULL argument");
    h->spec_cache.valid = false;
    h->lao_cache.valid = false;
    size_t need = 0;
    pt_checkpoint(h, nullptr, &need);
    if (len != need) return fail(h, PT_ERR_ARG, "checkpoint size does not match this handle");
    const uint8_t* p = static_cast<const uint8_t*>(buf);
    int64_t hdr[8];
    std::memcpy(hdr, p, 64);
    if (hdr[0] != 0x5054434bLL || hdr[1] != h->L || hdr[2] != h->NT || hdr[3] != h->R)
        return fail(h, PT_ERR_ARG, "checkpoint shape does not match this handle");
    p += 64;
    for (int e = 0; e < h->n_edges; ++e)
        if ((int8_t)p[e] < -J_ABS_MAX) return fail(h, PT_ERR_ARG, "corrupt couplers in checkpoint");
    {
        const int km = coupler_kmax(h->L, reinterpret_cast<const int8_t*>(p));
        if (km > KT_MAX - 1) return fail(h, PT_ERR_ARG, "corrupt couplers in checkpoint");
        if (int rc0 = ensure_table_rows(h, km)) return rc0;
    }
    Group& g = h->main;
    const size_t reps = (size_t)h->R * h->NT, npair = (size_t)h->R * (h->NT > 1 ? h->NT - 1 : 1);
    {
        // the kernels index tables by local field and buffers by slot map:
        // spins must be +-1 and every run's map a permutation of the slots
        const int8_t* sp = reinterpret_cast<const int8_t*>(p + h->n_edges);
        for (size_t i = 0; i < reps * h->N; ++i)
            if (sp[i] != 1 && sp[i] != -1) return fail(h, PT_ERR_ARG, "corrupt spins in checkpoint");
        const uint8_t* pm = p + h->n_edges + reps * h->N + 4 * reps;
        for (int r = 0; r < h->R; ++r) {
            uint64_t seen = 0;
            for (int t = 0; t < h->NT; ++t) {
                const int b = pm[(size_t)r * h->NT + t];
                if (b >= h->NT || (seen >> b & 1ull)) return fail(h, PT_ERR_ARG, "corrupt slot map in checkpoint");
                seen |= 1ull << b;
            }
        }
    }
    h->J.assign(reinterpret_cast<const int8_t*>(p), reinterpret_cast<const int8_t*>(p) + h->n_edges);
    p += h->n_edges;
    int rc = upload_couplers(h, g, 0, h->J.data());
    if (rc) return rc;
    g.sweep = (uint64_t)hdr[4];
    h->uid = (uint32_t)hdr[5];
    g.desc[0].uid = h->uid;
    if ((rc = upload_desc(h, g))) return rc;
    CK(cudaMemcpyAsync(g.spins, p, reps * h->N, cudaMemcpyHostToDevice, h->stream), "restore spins"); p += reps * h->N;
    CK(cudaMemcpyAsync(g.E, p, 4 * reps, cudaMemcpyHostToDevice, h->stream), "restore E"); p += 4 * reps;
    CK(cudaMemcpyAsync(g.perm, p, reps, cudaMemcpyHostToDevice, h->stream), "restore perm"); p += reps;
    CK(cudaMemcpyAsync(g.best, p, 4 * (size_t)h->R, cudaMemcpyHostToDevice, h->stream), "restore best"); p += 4 * (size_t)h->R;
    CK(cudaMemcpyAsync(g.first, p, 4 * (size_t)h->R, cudaMemcpyHostToDevice, h->stream), "restore first"); p += 4 * (size_t)h->R;
    CK(cudaMemcpyAsync(g.macc, p, 8 * reps, cudaMemcpyHostToDevice, h->stream), "restore macc"); p += 8 * reps;
    CK(cudaMemcpyAsync(g.xacc, p, 8 * npair, cudaMemcpyHostToDevice, h->stream), "restore xacc");
    if ((rc = walk_clear(h, g))) return rc;  // the restored buffers start a new walk
    CK(cudaStreamSynchronize(h->stream), "sync restore");
    return PT_OK;
}

int pt_set_schedule(pt_handle* h, int32_t sp, int32_t ipc, int32_t spl)
{
    if (!h) return PT_ERR_ARG;
    const int nsp = sp > 0 ? sp : h->sp, nipc = ipc > 0 ? ipc : h->ipc;
    if (spl < 0) return fail(h, PT_ERR_ARG, "sweeps_per_launch must be >= 0");
    int rc = check_schedule(h, h->L, h->NT, nsp, nipc, h->team);
    if (rc) return rc;
    if ((rc = apply_schedule(h, h->team, nsp, nipc))) return rc;
    if (spl > 0) h->spl = spl;
    CK(cudaStreamSynchronize(h->stream), "sync schedule");
    return PT_OK;
}

int pt_set_mapping(pt_handle* h, int32_t team, int32_t slot_parallel, int32_t runs_per_cta)
{
    if (!h || team < 0) return fail(h, PT_ERR_ARG, "team must be >= 0");
    const int nsp = slot_parallel > 0 ? slot_parallel : h->sp, nipc = runs_per_cta > 0 ? runs_per_cta : h->ipc;
    int rc = check_schedule(h, h->L, h->NT, nsp, nipc, team);
    if (rc) return rc;
    if ((rc = apply_schedule(h, team, nsp, nipc))) return rc;
    CK(cudaStreamSynchronize(h->stream), "sync mapping");
    return PT_OK;
}

int pt_get_mapping(const pt_handle* h, int32_t* team)
{
    if (!h || !team) return PT_ERR_ARG;
    *team = h->team;
    return PT_OK;
}

int pt_set_walk_stats(pt_handle* h, int32_t on)
{
    if (!h) return PT_ERR_ARG;
    Group& g = h->main;
    const size_t reps = (size_t)g.n_inst * g.R * g.NT;
    if (on && !g.walk) {
        // the walk arrays enlarge each run's shared-memory block: check first
        int cap = 0;
        CK(sweep_smem_capacity(&cap), "shared memory capacity");
        if (bundle_smem_bytes(g.L, g.NT, h->ipc, h->team, true, h->kt) > cap)
            return fail(h, PT_ERR_ARG, "the current schedule leaves no shared memory for the walk counters");
        unsigned long long *whot = nullptr, *wtrips = nullptr;
        uint8_t* wstate = nullptr;
        cudaError_t e = dalloc(&whot, reps);
        if (e == cudaSuccess) e = dalloc(&wtrips, reps);
        if (e == cudaSuccess) e = dalloc(&wstate, reps);
        if (e != cudaSuccess) {                 // nothing half-allocated stays behind
            cudaFree(whot); cudaFree(wtrips); cudaFree(wstate);
            return cuda_fail(h, e, "cudaMalloc walk");
        }
        g.whot = whot; g.wtrips = wtrips; g.wstate = wstate;
        g.walk = true;
        for (int i = 0; i < g.n_inst; ++i) {
            const size_t r0 = (size_t)i * g.R * g.NT;
            g.desc[i].whot = g.whot + r0;
            g.desc[i].wtrips = g.wtrips + r0;
            g.desc[i].wstate = g.wstate + r0;
        }
    } else if (!on && g.walk) {
        CK(cudaStreamSynchronize(h->stream), "sync walk");
        cudaFree(g.whot); cudaFree(g.wtrips); cudaFree(g.wstate);
        g.whot = g.wtrips = nullptr;
        g.wstate = nullptr;
        g.walk = false;
        for (auto& d : g.desc) d.whot = d.wtrips = nullptr, d.wstate = nullptr;
    }
    int rc = upload_desc(h, g);
    if (!rc) rc = group_schedule(h, g);
    if (rc && g.walk && on) {
        // the walk kernels need the enlarged shared-memory block of the new
        // schedule: without it, go back to untracked runs
        cudaStreamSynchronize(h->stream);
        cudaFree(g.whot); cudaFree(g.wtrips); cudaFree(g.wstate);
        g.whot = g.wtrips = nullptr;
        g.wstate = nullptr;
        g.walk = false;
        for (auto& d : g.desc) d.whot = d.wtrips = nullptr, d.wstate = nullptr;
        const std::string why = h->err;
        upload_desc(h, g);
        h->err = why;
        return rc;
    }
    if (!rc) rc = walk_clear(h, g);
    if (rc) return rc;
    CK(cudaStreamSynchronize(h->stream), "sync walk");
    return PT_OK;
}

int pt_get_walk_stats(pt_handle* h, uint64_t* hot, uint64_t* trips, uint64_t* n_passes)
{
    if (!h) return PT_ERR_ARG;
    Group& g = h->main;
    if (!g.walk) return fail(h, PT_ERR_STATE, "the walk is not tracked (pt_set_walk_stats)");
    const size_t reps = (size_t)g.R * g.NT;
    if (hot) CK(cudaMemcpyAsync(hot, g.whot, 8 * reps, cudaMemcpyDeviceToHost, h->stream), "download walk");
    if (trips) CK(cudaMemcpyAsync(trips, g.wtrips, 8 * reps, cudaMemcpyDeviceToHost, h->stream), "download walk");
    CK(cudaStreamSynchronize(h->stream), "sync walk");
    if (n_passes) *n_passes = g.walk_passes;
    return PT_OK;
}

// Times candidate schedules on a batch of `n_inst` copies of this instance
// (the speculative engineering batch) and keeps the fastest.  Candidates: every
// slot_parallel with slot_parallel * L^2 a multiple of 32 and at most 1024
// threads, with runs per CTA 1, 2 or 4 (shared memory permitting).  The
// candidate batch is left in an unspecified state; the main runs are untouched.
int pt_autotune(pt_handle* h, int32_t n_inst, int32_t trial_sweeps)
{
    if (!h || n_inst < 1 || n_inst > 16 || trial_sweeps < 1) return fail(h, PT_ERR_ARG, "need 1 <= n_inst <= 16, trial_sweeps >= 1");
    int rc = ensure_candidates(h, n_inst);
    if (rc) return rc;
    Group& g = h->cand;
    for (int j = 0; j < g.n_inst; ++j) {
        int r2 = upload_couplers(h, g, j, h->J.data());
        if (r2) return r2;
        g.desc[j].uid = 0x7A11u + (uint32_t)j;
    }
    if ((rc = upload_desc(h, g))) return rc;
    if ((rc = group_reset(h, g, true))) return rc;
    const int L2 = h->L * h->L;
    int cap = 0;
    CK(sweep_smem_capacity(&cap), "shared memory capacity");
    const int old_sp = h->sp, old_ipc = h->ipc, old_team = h->team;
    const bool old_timing = h->timing;
    h->timing = true;
    double best_rate = 0.0;
    int best_sp = old_sp, best_ipc = old_ipc, best_team = old_team;
    // candidate (team, slot_parallel) pairs: cell-major (team 0) and slot-major
    std::vector<std::pair<int, int>> cands;
    for (int sp = 1; sp <= h->NT && sp * L2 <= MAX_THREADS; ++sp)
        if ((sp * L2) % 32 == 0) cands.push_back({0, sp});
    for (int team : {2, 4, 8, 16, 32}) {
        if (team > L2) break;
        for (int nt : {h->NT, (h->NT + 1) / 2, (h->NT + 3) / 4, (h->NT + 7) / 8})
            if (nt >= 1 && nt * team >= 32 && nt * team <= MAX_THREADS_SM) cands.push_back({team, nt});
    }
    for (const auto& c : cands) {
        const int team = c.first, sp = c.second;
        const int tpr = team > 0 ? sp * team : sp * L2;
        for (int ipc : {1, 2, 4}) {
            if (tpr * ipc > (team > 0 ? MAX_THREADS_SM : MAX_THREADS) || ipc > h->R) break;
            if (bundle_smem_bytes(h->L, h->NT, ipc, team, false, h->kt) > cap) break;
            h->team = team;
            h->sp = sp;
            h->ipc = ipc;
            if (!(rc = group_schedule(h, g))) rc = group_sweeps(h, g, trial_sweeps, 1);
            if (rc) {
                h->timing = old_timing;
                h->team = old_team; h->sp = old_sp; h->ipc = old_ipc;
                return rc;
            }
            CK(cudaStreamSynchronize(h->stream), "sync autotune");
            double ms = 0.0;
            for (int i = 0; i < h->ev_used; ++i) {
                float t = 0.f;
                CK(cudaEventElapsedTime(&t, h->ev[2 * i], h->ev[2 * i + 1]), "event time");
                ms += t;
            }
            const double rate = (double)g.n_inst * h->R * h->NT * h->N * trial_sweeps / (ms * 1e-3);
            if (rate > best_rate) { best_rate = rate; best_sp = sp; best_ipc = ipc; best_team = team; }
        }
    }
    h->timing = old_timing;
    h->team = old_team; h->sp = old_sp; h->ipc = old_ipc;
    if ((rc = apply_schedule(h, best_team, best_sp, best_ipc))) return rc;
    CK(cudaStreamSynchronize(h->stream), "sync autotune");
    return PT_OK;
}

int pt_get_schedule(const pt_handle* h, int32_t* sp, int32_t* ipc, int32_t* spl)
{
    if (!h) return PT_ERR_ARG;
    if (sp) *sp = h->sp;
    if (ipc) *ipc = h->ipc;
    if (spl) *spl = h->spl;
    return PT_OK;
}

uint64_t pt_launch_count(const pt_handle* h) { return h ? h->launches : 0; }

int pt_select_device(int32_t device)
{
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDeviceCount");
    if (device < 0 || device >= n) return fail(nullptr, PT_ERR_ARG, "device index out of range");
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaSetDevice");
    return PT_OK;
}

int pt_set_timing(pt_handle* h, int on)
{
    if (!h) return PT_ERR_ARG;
    h->timing = on != 0;
    h->total_ms = 0.0;
    h->total_launches = 0;
    return PT_OK;
}

int pt_sweep_timing_total(const pt_handle* h, double* ms, uint64_t* launches)
{
    if (!h) return PT_ERR_ARG;
    if (ms) *ms = h->total_ms;
    if (launches) *launches = h->total_launches;
    return PT_OK;
}

int pt_eval_stats(pt_handle* h, uint64_t* evals, uint64_t* batches, double* device_ms, int reset)
{
    if (!h) return PT_ERR_ARG;
    if (evals) *evals = h->evals;
    if (batches) *batches = h->batches;
    if (device_ms) *device_ms = h->eval_ms;
    if (reset) {
        h->evals = h->batches = 0;
        h->eval_ms = 0.0;
    }
    return PT_OK;
}

int pt_last_sweep_timing(const pt_handle* h, double* ms, int32_t* launches)
{
    if (!h) return PT_ERR_ARG;
    if (ms) *ms = h->last_ms;
    if (launches) *launches = h->last_launches;
    return PT_OK;
}

}  // extern "C"
