// pt_kernels.cu -- sm_103a kernels of the parallel-tempering hardness engine.
//
// Method (arXiv:1605.03607): Ising cost of Eq. 1 on the Chimera graph
// (Appendix A), parallel tempering of Sec. II (independent Metropolis updates,
// neighbour swaps with detailed-balance acceptance), sweeps as in Sec. III.B.
//
// Design (GB300):
//   * One CTA "bundle" = a few PT runs of one instance.  Every replica of those
//     runs lives in shared memory for the whole launch as int8 spins, one
//     32-bit word per group of 4 same-colour spins of a cell, colour-major.
//   * A thread owns one Chimera cell (its couplers, negated and packed for
//     dp4a, sit in 16 registers) and a strided subset of temperature slots.
//     Per group update: 4 shared loads, one Philox4x32-10 call for the 4
//     spins, 8 dp4a for the local fields, 4 table compares, 1 store.
//   * Energies are kept incrementally: per-lane dE and flip counts are packed
//     in one int, reduced with redux.sync (a warp spans at most two slots) and
//     added to the slot energy with one shared atomic.
//   * Replica exchange is fused: before each sweep one warp turns every pair's
//     uniform into the largest accepted half energy gap c_p (exact search of
//     the host-built table, which is non-increasing), so the serial ascending
//     swap chain is a subtract and compare per pair.
//   * No tensor cores: this is integer ALU / shared-memory work.
#include <atomic>
#include <climits>
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>

#include "pt_internal.h"
#include "pt_kernels.h"
#include "pt_philox.cuh"

namespace ptg {

// Debug builds (-DPT_DEBUG): every data-dependent shared or global index of
// the kernels below is checked.  A failed check records its code in a device
// word (the first failure wins) and the access goes to index 0 instead, so
// the kernel neither faults nor leaves a barrier early; the launchers then
// synchronise the stream and read the word (debug_check).  Codes:
//   1 Metropolis table row >= rows per slot     2 slot map entry >= n_temps
//   3 exchange table range outside the tables   4 run index >= runs
//   5 neighbour spin word outside the buffer    6 TTS over more than 1024 runs
//   7 energy kernel: slot map entry >= n_temps
//   8 closed-form exchange criterion differs from the table search
//   9 a bundle's lattice side differs from the kernel's compile-time side
// Release builds compile the checks away.
#ifdef PT_DEBUG
__device__ unsigned int g_pt_debug_code;
__device__ __forceinline__ int dbg_idx(int i, int n, unsigned code)
{
    if ((unsigned)i >= (unsigned)n) {
        atomicCAS(&g_pt_debug_code, 0u, code);
        return 0;
    }
    return i;
}
#define PT_IDX(i, n, code) ::ptg::dbg_idx((i), (n), (code))
#else
#define PT_IDX(i, n, code) (i)
#endif

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;

// Exact search of the exchange table from a start point c0 in [0, H]: the
// largest h in [0, H] with tab[h'] > u for all 1 <= h' <= h.  Exact for any
// start point because the table is non-increasing in h (checked on the host);
// both neighbours of the start are loaded at once.
__device__ __forceinline__ int half_gap_search(const uint32_t* tab, int H, uint32_t u, int c)
{
    const uint32_t at = c > 0 ? tab[c] : 0xFFFFFFFFu;
    const uint32_t above = c < H ? tab[c + 1] : 0u;
    if (c > 0 && at <= u) {
        --c;
        while (c > 0 && tab[c] <= u) --c;
    } else if (c < H && above > u) {
        ++c;
        while (c < H && tab[c + 1] > u) ++c;
    }
    return c;
}

// Critical half-gap c_p of pair p for the uniform u: a swap with energy gap
// d = 2h > 0 is accepted iff h <= c_p, where c_p is the number of table
// entries xthr[p][h] = floor(2^32 exp(-2 h dbeta_p)) (h = 1..H_p) above u.
// Such an entry exceeds u iff 2^32 exp(-2 h dbeta_p) >= u + 1, i.e. iff
// h <= X = log2(2^32 / (u + 1)) * ln2 / (2 dbeta_p), so c_p = min(H_p, floor X).
// X is evaluated in single precision from the hint ln2 / (2 dbeta_p):
// log2f is accurate to 1 ulp of its result (at most X * 2^-23 after the
// product), the argument u + 1 (or u for u >= 2^24, off by at most 2^-23 in
// log2) and the hint and product roundings (2^-24 each) add at most
// X * 1.2e-7 + hint * 1.8e-7, and the host's FP64 tables round 1e-14
// relative.  When X lies further than twice that bound from an integer the
// floor is exact and no table entry is read; otherwise (a few times in 10^5)
// the table is searched, from a separate fast-intrinsic estimate (any start
// point gives the exact result; keeping the first estimate live through the
// search measured 1 % slower).  Debug builds also search on the closed-form
// path and record code 8 if the two ever differ.
__device__ __forceinline__ int critical_half_gap(const InstDesc& in, const int32_t* xoff_sm,
                                                 const float* xhint_sm, int p, uint32_t u)
{
    const int o = xoff_sm[p];
#ifdef PT_DEBUG
    const int total = xoff_sm[in.NT - 1];
    const int H = (o < 0 || xoff_sm[p + 1] < o || xoff_sm[p + 1] > total)
                      ? (atomicCAS(&g_pt_debug_code, 0u, 3u), 0) : xoff_sm[p + 1] - o;
#else
    const int H = xoff_sm[p + 1] - o;
#endif
    const uint32_t* tab = in.xthr + o - 1;       // tab[h], h = 1..H
    if (u == 0u) return H;                       // every entry is >= 1
    const float hint = xhint_sm[p];
    const float x = u < (1u << 24) ? (float)(u + 1u) : (float)u;
    const float est = -log2f(x * 0x1p-32f) * hint;
    const float eps = est * 8e-7f + hint * 4e-7f + 2e-6f;
    if (est >= (float)H + eps) {
#ifdef PT_DEBUG
        if (half_gap_search(tab, H, u, H) != H) atomicCAS(&g_pt_debug_code, 0u, 8u);
#endif
        return H;
    }
    const float fl = floorf(est);
    if (est < (float)H && est - fl > eps && (fl + 1.0f) - est > eps) {
#ifdef PT_DEBUG
        if (half_gap_search(tab, H, u, (int)fl) != (int)fl) atomicCAS(&g_pt_debug_code, 0u, 8u);
#endif
        return (int)fl;
    }
    const float start = (32.0f - __log2f((float)u)) * xhint_sm[p];
    return half_gap_search(tab, H, u, start <= 0.0f ? 0 : (start >= (float)H ? H : (int)start));
}

struct CellRegs {
    uint32_t jin[4], jud[4];
    int own, opp, mn, pl;   // word offsets inside one buffer
    uint32_t gidx;          // natural group index i >> 2 of the group
};

__device__ __forceinline__ void load_cell(const InstDesc& in, int q, int col, int L2, int L,
                                          CellRegs& cr)
{
    const uint32_t* jw = in.jw + (q * 2 + col) * 8;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        cr.jin[k] = jw[k];
        cr.jud[k] = jw[4 + k];
    }
    const int r = q / L, c = q - r * L;
    const int u = (r + c + col) & 1;
    cr.gidx = (uint32_t)(2 * q + u);
    cr.own = col * L2 + q;
    cr.opp = (1 - col) * L2 + q;
    cr.mn = (1 - col) * L2 + in.nbr[(q * 2 + col) * 2 + 0];
    cr.pl = (1 - col) * L2 + in.nbr[(q * 2 + col) * 2 + 1];
}

// Per-lane result of one group update, packed for one warp reduction:
// (sum of accepted k) * 1024 + popcount of the flip mask (7 bits per flip).
__device__ __forceinline__ void apply_packed(int32_t* Es, uint32_t* macc, int t, int v)
{
    const int pc = v & 1023;
    const int dk = (v - pc) >> 10;
    if (dk) atomicAdd(&Es[t], 2 * dk);
    if (pc) atomicAdd(&macc[t], (uint32_t)(pc / 7));
}

struct WarpSeg {
    bool two;        // the warp's lanes cover two slots
    bool lo;         // this lane belongs to the first of them
    int lane_hi;     // first lane of the second slot
    int sp_first;    // slot phase of lane 0
    bool redux;      // warp reduction usable (at most two slots per warp)
};

// One Metropolis half-sweep (one colour) over this thread's slots.
__device__ __forceinline__ void colour_phase(const CellRegs& cr, uint32_t* sw, int NW,
                                             const uint32_t* thr_sm, int kt, int32_t* Es, uint32_t* macc,
                                             const uint8_t* perm, int NT, int SP, int sp,
                                             int iters, uint32_t s, uint32_t runbits,
                                             uint32_t k0, uint32_t k1, const WarpSeg& ws, int lane)
{
    const PhiloxPre pre = philox_pre(s, cr.gidx, k0, k1);
    for (int i = 0; i < iters; ++i) {
        const int t = sp + i * SP;
        int packed = 0;
        if (t < NT) {
            uint32_t* bw = sw + PT_IDX((int)perm[t], NT, 2u) * NW;
            const uint32_t own = bw[cr.own];
            const int opp = (int)bw[cr.opp];
            const uint32_t mw = bw[PT_IDX(cr.mn, NW, 5u)], pw = bw[PT_IDX(cr.pl, NW, 5u)];
            const uint4 rn = philox_slot(pre, runbits | (uint32_t)t, k0, k1);
            const uint32_t* th = thr_sm + t * kt;
            const int x01 = (int)__byte_perm(mw, pw, 0x5140);
            const int x23 = (int)__byte_perm(mw, pw, 0x7362);
            // -h_i for the 4 spins (couplers are stored negated)
            const int h0 = __dp4a((int)cr.jin[0], opp, __dp4a((int)cr.jud[0], x01, 0));
            const int h1 = __dp4a((int)cr.jin[1], opp, __dp4a((int)cr.jud[1], x01, 0));
            const int h2 = __dp4a((int)cr.jin[2], opp, __dp4a((int)cr.jud[2], x23, 0));
            const int h3 = __dp4a((int)cr.jin[3], opp, __dp4a((int)cr.jud[3], x23, 0));
            // k_i = -s_i h_i, dE = 2 k_i; accept if k_i <= 0 or u < thr[slot][k_i]
            const int kk0 = (int)(int8_t)(own) * h0;
            const int kk1 = (int)(int8_t)(own >> 8) * h1;
            const int kk2 = (int)(int8_t)(own >> 16) * h2;
            const int kk3 = (int)(int8_t)(own >> 24) * h3;
            const bool a0 = (kk0 <= 0) | (rn.x < th[PT_IDX(max(kk0, 0), kt, 1u)]);
            const bool a1 = (kk1 <= 0) | (rn.y < th[PT_IDX(max(kk1, 0), kt, 1u)]);
            const bool a2 = (kk2 <= 0) | (rn.z < th[PT_IDX(max(kk2, 0), kt, 1u)]);
            const bool a3 = (kk3 <= 0) | (rn.w < th[PT_IDX(max(kk3, 0), kt, 1u)]);
            uint32_t flip = 0u;
            int dk = 0;
            if (a0) { flip |= 0x000000FEu; dk += kk0; }
            if (a1) { flip |= 0x0000FE00u; dk += kk1; }
            if (a2) { flip |= 0x00FE0000u; dk += kk2; }
            if (a3) { flip |= 0xFE000000u; dk += kk3; }
            if (flip) bw[cr.own] = own ^ flip;
            packed = dk * 1024 + __popc(flip);
        }
        if (ws.redux) {
            if (ws.two) {
                const int lo = __reduce_add_sync(FULL, ws.lo ? packed : 0);
                const int hi = __reduce_add_sync(FULL, ws.lo ? 0 : packed);
                if (lane == 0 && lo) apply_packed(Es, macc, ws.sp_first + i * SP, lo);
                if (lane == ws.lane_hi && hi) apply_packed(Es, macc, ws.sp_first + 1 + i * SP, hi);
            } else {
                const int v = __reduce_add_sync(FULL, packed);
                if (lane == 0 && v) apply_packed(Es, macc, ws.sp_first + i * SP, v);
            }
        } else if (packed) {
            apply_packed(Es, macc, t, packed);
        }
    }
}

// Exchange critical gaps of every pair of this run for sweep counter s
// (called by one group of 32 threads; lane l handles pairs l and l + 32, the
// four lanes of pairs 4c..4c+3 each forming the Philox call c and taking its
// own word).  Table offsets and search hints come from shared memory.
__device__ __forceinline__ void exchange_prepare(const InstDesc& in, const uint32_t* thr_sm, int lane,
                                                 uint32_t s, uint32_t runbits, uint32_t k0, uint32_t k1,
                                                 int NT, int32_t* cc)
{
    // bundle tables: thr [NT][kt], then exchange offsets [NT] and search hints [NT]
    const int32_t* xoff_sm = reinterpret_cast<const int32_t*>(thr_sm + NT * in.kt);
    const float* xhint_sm = reinterpret_cast<const float*>(thr_sm + NT * in.kt + NT);
    const int npairs = NT - 1;
    for (int p = lane; p < npairs; p += 32) {
        const uint4 w = philox10(s, runbits, (uint32_t)(p >> 2), 1u, k0, k1);
        const int e = p & 3;
        const uint32_t u = e == 0 ? w.x : e == 1 ? w.y : e == 2 ? w.z : w.w;
        cc[p] = critical_half_gap(in, xoff_sm, xhint_sm, p, u);
    }
}

// Temperature random walk, after one exchange pass of a run (one thread).
// Copies are the configuration buffers.  Every copy in the hot half (the
// NT/2 highest temperatures: slots NT - NT/2 .. NT-1) gets one more pass
// there.  A copy at the coldest slot completes a round trip if it reached the
// hottest slot since it last sat at the coldest one; states: 0 neither end
// seen yet, 1 coldest slot seen, 2 hottest slot seen after it.
__device__ __forceinline__ void walk_update(const uint8_t* perm, uint32_t* whot, uint32_t* wtr, uint8_t* wst,
                                            int NT)
{
    for (int t = NT - NT / 2; t < NT; ++t) whot[perm[t]] += 1u;
    const int c = perm[0];
    if (wst[c] == 2) wtr[c] += 1u;
    wst[c] = 1;
    const int h = perm[NT - 1];
    if (wst[h] == 1) wst[h] = 2;
}

// The ascending exchange sweep of one run (one thread): a configuration that
// wins pair p is carried on to pair p+1.  Slot energies, slot map and
// acceptance criteria are read in blocks of 4 ahead of the carried chain.
// With INV the inverse map (buffer -> slot) is rewritten along the way.
template <bool INV>
__device__ __forceinline__ int exchange_chain(int32_t* Es, uint8_t* perm, uint8_t* inv, uint32_t* xacc,
                                              const int32_t* cc, int NT)
{
    constexpr int B = 4;
    const int np = NT - 1;
    int ce = Es[0], cb = perm[0], m = ce;
    int nxe[B], nxb[B], nxt[B];
#pragma unroll
    for (int i = 0; i < B; ++i) {
        const bool v = i < np;
        nxe[i] = v ? Es[i + 1] : 0;
        nxb[i] = v ? perm[i + 1] : 0;
        nxt[i] = v ? nxe[i] - 2 * cc[i] : 0;
    }
    for (int p0 = 0; p0 < np; p0 += B) {
        int ne[B], nb[B], tt[B];
#pragma unroll
        for (int i = 0; i < B; ++i) {
            ne[i] = nxe[i];
            nb[i] = nxb[i];
            tt[i] = nxt[i];
        }
#pragma unroll
        for (int i = 0; i < B; ++i) {            // prefetch: indices > p0+B, never stored below
            const int q = p0 + B + i;
            const bool v = q < np;
            nxe[i] = v ? Es[q + 1] : 0;
            nxb[i] = v ? perm[q + 1] : 0;
            nxt[i] = v ? nxe[i] - 2 * cc[q] : 0;
        }
        int oe[B], ob[B];
        unsigned bits = 0u;
#pragma unroll
        for (int i = 0; i < B; ++i) {
            if (p0 + i < np) {
                m = min(m, ne[i]);
                const bool a = tt[i] <= ce;          // E_{p+1} - E_p <= 2 c_p
                oe[i] = a ? ne[i] : ce;
                ob[i] = a ? nb[i] : cb;
                ce = a ? ce : ne[i];
                cb = a ? cb : nb[i];
                bits |= (unsigned)a << i;
            }
        }
#pragma unroll
        for (int i = 0; i < B; ++i) {
            if (p0 + i < np) {
                Es[p0 + i] = oe[i];
                perm[p0 + i] = (uint8_t)ob[i];
                if (INV) inv[ob[i]] = (uint8_t)(p0 + i);
                xacc[p0 + i] += (bits >> i) & 1u;
            }
        }
    }
    Es[np] = ce;
    perm[np] = (uint8_t)cb;
    if (INV) inv[cb] = (uint8_t)np;
    return m;
}

// The same exchange sweep run by all 32 lanes of one warp (NT <= 64; lane l
// holds slots l and l + 32), with no serial recurrence.  A chain of accepted
// swaps that starts at slot i carries the energy E_i upward and ends at the
// first pair p >= i whose bound E_{p+1} - 2 c_p exceeds E_i (that pair is
// rejected, and the next chain starts at slot p + 1).  Each lane finds that
// end for its own slots from a bit mask of the bounds above its energy
// (independent compares); pointer doubling over "next start = end + 1" then
// collects the ends met from slot 0 on, which are exactly the pairs the
// ascending pass rejects.  The slot contents follow from the accepted-pair
// mask: after the pass slot s holds the old content of slot s+1 when pair s
// was accepted, and otherwise the configuration carried into s, which
// started at the lowest slot of the run of accepted pairs ending at pair s-1
// (s itself when pair s-1 was rejected).  The pair criteria cc of this sweep
// are overwritten with the bounds.  Returns the lowest slot energy.
template <bool INV>
__device__ __forceinline__ int exchange_chain_warp(int32_t* Es, uint8_t* perm, uint8_t* inv, uint32_t* xacc,
                                                   int32_t* cc, int NT, int lane)
{
    const int np = NT - 1;
    const bool two = NT > 32;                      // warp-uniform
    const int s1 = lane + 32;
    const int e0 = lane < NT ? Es[lane] : INT_MAX;
    const int e1 = (two && s1 < NT) ? Es[s1] : INT_MAX;
    const int m = __reduce_min_sync(FULL, min(e0, e1));
    if (lane < np) cc[lane] = Es[lane + 1] - 2 * cc[lane];
    if (two && s1 < np) cc[s1] = Es[s1 + 1] - 2 * cc[s1];
    __syncwarp();
    // pairs whose bound exceeds this lane's slot energies (slot s1 >= 32 needs
    // only pairs >= 32)
    uint32_t r0lo = 0u, r0hi = 0u, r1hi = 0u;
#pragma unroll
    for (int p = 0; p < 32; ++p)
        if (p < np) r0lo |= (uint32_t)(cc[p] > e0) << p;
    if (two) {
#pragma unroll
        for (int p = 32; p < 63; ++p)
            if (p < np) {
                const int t = cc[p];
                r0hi |= (uint32_t)(t > e0) << (p - 32);
                r1hi |= (uint32_t)(t > e1) << (p - 32);
            }
    }
    // end of a chain starting at each slot (np: it carries to the top slot);
    // J = next chain start, R = the rejected pair as a bit (slots >= NT: none)
    const unsigned long long q0 = (((unsigned long long)r0hi << 32) | r0lo) & (~0ull << lane);
    const unsigned long long q1 = ((unsigned long long)r1hi << 32) & (~0ull << (s1 & 63));
    const int end0 = q0 ? __ffsll((long long)q0) - 1 : np;
    const int end1 = (two && s1 < NT && q1) ? __ffsll((long long)q1) - 1 : np;
    int J0 = lane < NT ? end0 + 1 : NT;
    int J1 = (two && s1 < NT) ? end1 + 1 : NT;
    unsigned long long R0 = (lane < NT && end0 < np) ? 1ull << end0 : 0ull;
    unsigned long long R1 = (two && s1 < NT && end1 < np) ? 1ull << end1 : 0ull;
    // doubling: after k rounds R holds the rejections of the next 2^k chains
    for (int k = 0; (1 << k) < NT; ++k) {
        const int a = J0 < NT ? J0 : 0, b = J1 < NT ? J1 : 0;
        unsigned long long Ra, Rb = 0ull;
        int Ja, Jb = NT;
        if (two) {
            const unsigned long long Ra0 = __shfl_sync(FULL, R0, a & 31), Ra1 = __shfl_sync(FULL, R1, a & 31);
            const unsigned long long Rb0 = __shfl_sync(FULL, R0, b & 31), Rb1 = __shfl_sync(FULL, R1, b & 31);
            const int Ja0 = __shfl_sync(FULL, J0, a & 31), Ja1 = __shfl_sync(FULL, J1, a & 31);
            const int Jb0 = __shfl_sync(FULL, J0, b & 31), Jb1 = __shfl_sync(FULL, J1, b & 31);
            Ra = a >= 32 ? Ra1 : Ra0;
            Rb = b >= 32 ? Rb1 : Rb0;
            Ja = a >= 32 ? Ja1 : Ja0;
            Jb = b >= 32 ? Jb1 : Jb0;
        } else {                                   // NT <= 32: one slot per lane, pairs < 32
            Ra = (unsigned long long)__shfl_sync(FULL, (uint32_t)R0, a);
            Ja = __shfl_sync(FULL, J0, a);
        }
        if (J0 < NT) { R0 |= Ra; J0 = Ja; }
        if (J1 < NT) { R1 |= Rb; J1 = Jb; }
    }
    const unsigned long long mask = ~__shfl_sync(FULL, R0, 0) & ((1ull << np) - 1ull);
    // every slot's new content from the mask, gathered before any slot is rewritten
    int e_new[2] = {0, 0}, b_new[2] = {0, 0};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int s = lane + 32 * h;
        if (s < NT) {
            int src;
            if (s < np && ((mask >> s) & 1ull)) {
                src = s + 1;
            } else {
                const unsigned long long below = ~mask & ((1ull << s) - 1ull);
                src = below ? 64 - __clzll((long long)below) : 0;
            }
            e_new[h] = Es[src];
            b_new[h] = perm[src];
        }
    }
    __syncwarp();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int s = lane + 32 * h;
        if (s < NT) {
            Es[s] = e_new[h];
            perm[s] = (uint8_t)b_new[h];
            if (INV) inv[b_new[h]] = (uint8_t)s;
            if (s < np) xacc[s] += (uint32_t)((mask >> s) & 1ull);
        }
    }
    __syncwarp();
    return m;
}

// Lowest slot energy of a run, by all 32 lanes of one warp.
__device__ __forceinline__ int slot_min_warp(const int32_t* Es, int NT, int lane)
{
    int m = INT_MAX;
    for (int t = lane; t < NT; t += 32) m = min(m, Es[t]);
    return __reduce_min_sync(FULL, m);
}

template <bool WALK>
__device__ void process_bundle(const InstDesc* __restrict__ insts, const Bundle bd,
                               uint32_t sweep0, int nsweeps, int xevery, int mode,
                               unsigned char* smem)
{
    const InstDesc& in = insts[bd.inst];
    const int L = in.L, NT = in.NT, L2 = L * L, N = 8 * L2, NW = N / 4;
    const int SP = bd.sp, TPI = SP * L2;
    const int tid = threadIdx.x;
    const int item = tid / TPI, j = tid - item * TPI;
    const bool active = item < bd.nitems;
    const int q = j % L2, sp = j / L2;
    const int run = PT_IDX(bd.run0 + (active ? item : 0), in.R, 4u);
    constexpr bool walk = WALK;
    const ItemLayout lay = item_layout(L, NT, 0, walk);

    // bundle tables: thr [NT][kt], then exchange offsets [NT] and search hints [NT]
    const int KTI = in.kt;
    uint32_t* thr_sm = reinterpret_cast<uint32_t*>(smem);
    unsigned char* ib = smem + table_bytes(NT, KTI) + (active ? item : 0) * lay.bytes;
    uint32_t* sw = reinterpret_cast<uint32_t*>(ib + lay.spins);
    int32_t* Es = reinterpret_cast<int32_t*>(ib + lay.E);
    int32_t* ccrit = reinterpret_cast<int32_t*>(ib + lay.ccrit);     // 2 x NT, by sweep parity
    uint32_t* macc = reinterpret_cast<uint32_t*>(ib + lay.macc);
    uint32_t* xacc = reinterpret_cast<uint32_t*>(ib + lay.xacc);
    uint8_t* perm = ib + lay.perm;
    int32_t* misc = reinterpret_cast<int32_t*>(ib + lay.misc);

    // ---- load the instance table and this bundle's runs into shared memory
    for (int w = tid; w < NT * KTI; w += blockDim.x) thr_sm[w] = in.thr[w];
    for (int p = tid; p < NT; p += blockDim.x) {
        reinterpret_cast<int32_t*>(thr_sm + NT * KTI)[p] = in.xoff[p];
        reinterpret_cast<float*>(thr_sm + NT * KTI + NT)[p] = p < NT - 1 ? in.xhint[p] : 0.0f;
    }
    const size_t rep0 = (size_t)run * NT;
    if (active) {
        const uint32_t* gsp = reinterpret_cast<const uint32_t*>(in.spins + rep0 * N);
        for (int w = j; w < NT * NW; w += TPI) {
            const int buf = w / NW, g = w - buf * NW;
            const int cell = g >> 1, u = g & 1, r = cell / L, c = cell - r * L;
            sw[buf * NW + ((r + c + u) & 1) * L2 + cell] = gsp[w];
        }
        for (int t = j; t < NT; t += TPI) {
            Es[t] = in.E[rep0 + t];
            perm[t] = in.perm[rep0 + t];
            macc[t] = 0u;
            xacc[t] = 0u;
            if (walk) {
                reinterpret_cast<uint32_t*>(ib + lay.whot)[t] = 0u;
                reinterpret_cast<uint32_t*>(ib + lay.wtrips)[t] = 0u;
                (ib + lay.wstate)[t] = in.wstate[rep0 + t];
            }
        }
        if (j == 0) {
            misc[0] = in.best[run];
            misc[1] = in.first[run];
        }
    }

    // couplers of the colour about to be updated; the other colour's are
    // loaded right after each phase so the load latency hides behind the barrier
    CellRegs cr;
    if (active) load_cell(in, q, 0, L2, L, cr);
    const int lane = tid & 31;
    WarpSeg ws;
    ws.sp_first = __shfl_sync(FULL, sp, 0);
    ws.lo = (sp == ws.sp_first);
    const unsigned hi_mask = __ballot_sync(FULL, !ws.lo);
    ws.two = hi_mask != 0u;
    ws.lane_hi = ws.two ? __ffs(hi_mask) - 1 : 32;
    // warp reductions need a full warp of one run spanning at most two slots
    // (true for L^2 >= 32 or L^2 == 16 with whole warps per run); otherwise
    // every lane adds its own result atomically
    const unsigned act_mask = __ballot_sync(FULL, active);
    const bool one_item = __shfl_sync(FULL, item, 0) == __shfl_sync(FULL, item, 31);
    ws.redux = ((L2 >= 32) || (L2 == 16 && TPI % 32 == 0)) && act_mask == FULL && one_item;
    const int iters = (NT + SP - 1) / SP;
    // read through a warp reduction: the keys (and every Philox round key and
    // per-sweep product derived from them) are then warp-uniform values
    const uint32_t k0 = __reduce_or_sync(FULL, in.seed), k1 = __reduce_or_sync(FULL, in.uid);
    const uint32_t runbits = (uint32_t)run << 16;
    const int prep_warp_j0 = TPI - 32;          // last warp of the run prepares exchanges
    // a run whose threads start on a warp boundary passes its exchange chain
    // with its first warp; otherwise one thread does
    const bool warp_pass = ((item * TPI) & 31) == 0;
    auto exch = [&](uint32_t sw_) {
        return (NT > 1) && ((mode == 1) || (xevery > 0 && (sw_ % (uint32_t)xevery) == 0u));
    };
    const int n_iter = (mode == 0) ? nsweeps : 1;
    const uint32_t s_first = (mode == 0) ? sweep0 + 1u : sweep0;
    __syncthreads();                            // tables staged before the first exchange preparation
    if (n_iter > 0 && exch(s_first) && active && j >= prep_warp_j0)
        exchange_prepare(in, thr_sm, j - prep_warp_j0, s_first, runbits, k0, k1, NT, ccrit + (s_first & 1u) * NT);
    __syncthreads();

    for (int it = 0; it < n_iter; ++it) {
        const uint32_t s = s_first + (uint32_t)it;
        const bool do_x = exch(s);
        if (mode == 0) {
            if (active) {
                colour_phase(cr, sw, NW, thr_sm, KTI, Es, macc, perm, NT, SP, sp, iters, s, runbits,
                             k0, k1, ws, lane);
                load_cell(in, q, 1, L2, L, cr);
            }
            __syncthreads();
            if (active) {
                colour_phase(cr, sw, NW, thr_sm, KTI, Es, macc, perm, NT, SP, sp, iters, s, runbits,
                             k0, k1, ws, lane);
                load_cell(in, q, 0, L2, L, cr);
            }
        }
        __syncthreads();
        if (active && (warp_pass ? j < 32 : j == 0)) {
            int m;
            if (do_x) {
                m = warp_pass ? exchange_chain_warp<false>(Es, perm, nullptr, xacc, ccrit + (s & 1u) * NT, NT, j)
                              : exchange_chain<false>(Es, perm, nullptr, xacc, ccrit + (s & 1u) * NT, NT);
                if (WALK && j == 0)
                    walk_update(perm, reinterpret_cast<uint32_t*>(ib + lay.whot),
                                reinterpret_cast<uint32_t*>(ib + lay.wtrips), ib + lay.wstate, NT);
            } else if (warp_pass) {
                m = slot_min_warp(Es, NT, j);
            } else {
                m = Es[0];
                for (int p = 1; p < NT; ++p) m = min(m, Es[p]);
            }
            if (j == 0 && mode == 0 && m < misc[0]) {
                misc[0] = m;
                misc[1] = (int32_t)s;
            }
        }
        // meanwhile the last warp prepares the next sweep's exchange criteria
        if (it + 1 < n_iter && exch(s + 1u) && active && j >= prep_warp_j0)
            exchange_prepare(in, thr_sm, j - prep_warp_j0, s + 1u, runbits, k0, k1, NT, ccrit + ((s + 1u) & 1u) * NT);
        __syncthreads();
    }

    // ---- write the state back
    if (active) {
        uint32_t* gsp = reinterpret_cast<uint32_t*>(in.spins + rep0 * N);
        for (int w = j; w < NT * NW; w += TPI) {
            const int buf = w / NW, g = w - buf * NW;
            const int cell = g >> 1, u = g & 1, r = cell / L, c = cell - r * L;
            gsp[w] = sw[buf * NW + ((r + c + u) & 1) * L2 + cell];
        }
        for (int t = j; t < NT; t += TPI) {
            in.E[rep0 + t] = Es[t];
            in.perm[rep0 + t] = perm[t];
            in.macc[rep0 + t] += macc[t];
            if (t < NT - 1) in.xacc[(size_t)run * (NT > 1 ? NT - 1 : 1) + t] += xacc[t];
            if (walk) {
                in.whot[rep0 + t] += reinterpret_cast<const uint32_t*>(ib + lay.whot)[t];
                in.wtrips[rep0 + t] += reinterpret_cast<const uint32_t*>(ib + lay.wtrips)[t];
                in.wstate[rep0 + t] = (ib + lay.wstate)[t];
            }
        }
        if (j == 0) {
            in.best[run] = misc[0];
            in.first[run] = misc[1];
        }
    }
    __syncthreads();
}

// One colour-`col` word (4 spins, cell q) of the slot-major update at the
// temperature of the slot whose threshold row is `th`: local fields from the
// cell record (dp4a over int8 couplers and spins), Metropolis test of each
// spin against its uniform in `rn`, the word written back (unchanged where
// nothing flipped: in a colour phase only the other colour's words are
// read), energy change and flip count accumulated (pc: -2 per flipped spin).
__device__ __forceinline__ void sm_word(const uint32_t* rec, uint4 meta, uint32_t* bw, int col, int L2, int q,
                                        const uint4 rn, const uint32_t* th, int kt, int& dk, int& pc)
{
    const uint4 jin = *reinterpret_cast<const uint4*>(rec);
    const uint4 jud = *reinterpret_cast<const uint4*>(rec + 4);
    const int ow = col * L2 + q;
    const uint32_t own = bw[ow];
    const int opp = (int)bw[(1 - col) * L2 + q];
    const uint32_t mw = bw[PT_IDX((int)meta.y, 2 * L2, 5u)], pw = bw[PT_IDX((int)meta.z, 2 * L2, 5u)];
    const int x01 = (int)__byte_perm(mw, pw, 0x5140);
    const int x23 = (int)__byte_perm(mw, pw, 0x7362);
    const int h0 = __dp4a((int)jin.x, opp, __dp4a((int)jud.x, x01, 0));
    const int h1 = __dp4a((int)jin.y, opp, __dp4a((int)jud.y, x01, 0));
    const int h2 = __dp4a((int)jin.z, opp, __dp4a((int)jud.z, x23, 0));
    const int h3 = __dp4a((int)jin.w, opp, __dp4a((int)jud.w, x23, 0));
    const int kk0 = (int)(int8_t)(own) * h0;
    const int kk1 = (int)(int8_t)(own >> 8) * h1;
    const int kk2 = (int)(int8_t)(own >> 16) * h2;
    const int kk3 = (int)(int8_t)(own >> 24) * h3;
    const bool a0 = (kk0 <= 0) | (rn.x < th[PT_IDX(max(kk0, 0), kt, 1u)]);
    const bool a1 = (kk1 <= 0) | (rn.y < th[PT_IDX(max(kk1, 0), kt, 1u)]);
    const bool a2 = (kk2 <= 0) | (rn.z < th[PT_IDX(max(kk2, 0), kt, 1u)]);
    const bool a3 = (kk3 <= 0) | (rn.w < th[PT_IDX(max(kk3, 0), kt, 1u)]);
    uint32_t flip = 0u;
    if (a0) { flip |= 0x000000FEu; dk += kk0; }
    if (a1) { flip |= 0x0000FE00u; dk += kk1; }
    if (a2) { flip |= 0x00FE0000u; dk += kk2; }
    if (a3) { flip |= 0xFE000000u; dk += kk3; }
    bw[ow] = own ^ flip;                           // unconditional: one compare fewer per word
    pc = __dp4a((int)flip, 0x01010101, pc);        // -2 per flipped spin (a flipped byte is 0xFE)
}

// Slot-major mapping: a team of G lanes (a power of two, inside one warp)
// owns every sp-th spin buffer of a run and updates it at the temperature of
// the slot that buffer currently sits in (inverse slot map); its lanes split
// the cells.  For each owned buffer the team updates colour 0, syncs the
// team, updates colour 1, and reduces its energy change and flip count once.
// Teams never wait for each other inside a sweep; the run's threads meet only
// around the exchange.  The random numbers stay indexed by (sweep, run, slot,
// group), so which team does the work does not change any result.
// Bank layout: buffer strides are congruent to G modulo 32 and the cell
// records are colour-major with a 48-byte stride, so a warp's own/opposite
// spin words and coupler records come without bank conflicts.
template <bool WALK, int LT>
__device__ void process_bundle_sm(const InstDesc* __restrict__ insts, const Bundle bd,
                                  uint32_t sweep0, int nsweeps, int xevery, int mode,
                                  unsigned char* smem)
{
    const InstDesc& in = insts[bd.inst];
    const int G = bd.team, NTEAM = bd.sp, TPI = G * NTEAM;
    // LT > 0: the lattice side is a compile-time constant (the launcher picks the
    // instantiation from the one L of every bundle in the launch), so every
    // offset derived from L folds into the instructions
#ifdef PT_DEBUG
    if (LT && in.L != LT) {                     // uniform per CTA: the whole CTA skips the bundle
        if (threadIdx.x == 0) atomicCAS(&g_pt_debug_code, 0u, 9u);
        return;
    }
#endif
    const int L = LT ? LT : in.L, NT = in.NT, L2 = L * L, N = 8 * L2, NW = N / 4, NWP = NW + sm_pad(L, G);
    const int tid = threadIdx.x;
    const int item = tid / TPI, j = tid - item * TPI;
    const bool active = item < bd.nitems;
    const int team = j / G, tl = j - team * G;
    const int run = PT_IDX(bd.run0 + (active ? item : 0), in.R, 4u);
    constexpr bool walk = WALK;
    const ItemLayout lay = item_layout(L, NT, sm_pad(L, G), walk);

    const int KTI = in.kt;
    uint32_t* thr_sm = reinterpret_cast<uint32_t*>(smem);
    uint32_t* rec_sm = reinterpret_cast<uint32_t*>(smem + table_bytes(NT, KTI));   // [2][L2][CELL_REC]
    unsigned char* ib = smem + table_bytes(NT, KTI) + cell_table_bytes(L) + (active ? item : 0) * lay.bytes;
    uint32_t* sw = reinterpret_cast<uint32_t*>(ib + lay.spins);
    int32_t* Es = reinterpret_cast<int32_t*>(ib + lay.E);
    int32_t* ccrit = reinterpret_cast<int32_t*>(ib + lay.ccrit);
    uint32_t* macc = reinterpret_cast<uint32_t*>(ib + lay.macc);
    uint32_t* xacc = reinterpret_cast<uint32_t*>(ib + lay.xacc);
    uint8_t* perm = ib + lay.perm;
    uint8_t* inv = ib + lay.inv;
    int32_t* misc = reinterpret_cast<int32_t*>(ib + lay.misc);

    // ---- tables, couplers, per-group offsets and this bundle's runs
    for (int w = tid; w < NT * KTI; w += blockDim.x) thr_sm[w] = in.thr[w];
    for (int p = tid; p < NT; p += blockDim.x) {
        reinterpret_cast<int32_t*>(thr_sm + NT * KTI)[p] = in.xoff[p];
        reinterpret_cast<float*>(thr_sm + NT * KTI + NT)[p] = p < NT - 1 ? in.xhint[p] : 0.0f;
    }
    for (int w = tid; w < L2 * 4; w += blockDim.x) {  // global: [cell][colour][in 4 | inter 4]
        const int qc = w >> 1, half = w & 1, q = qc >> 1, col = qc & 1;
        const uint4 v = reinterpret_cast<const uint4*>(in.jw)[w];
        *reinterpret_cast<uint4*>(rec_sm + (col * L2 + q) * CELL_REC + 4 * half) = v;
    }
    for (int w = tid; w < L2 * 2; w += blockDim.x) {
        const int q = w >> 1, col = w & 1, r = q / L, c = q - r * L;
        const uint32_t gidx = (uint32_t)(2 * q + ((r + c + col) & 1));
        const uint64_t gprod = (uint64_t)PHILOX_M1 * gidx;   // Philox round 0, word 2: fixed per cell
        const uint32_t mn = (uint32_t)((1 - col) * L2 + in.nbr[w * 2 + 0]);
        const uint32_t pl = (uint32_t)((1 - col) * L2 + in.nbr[w * 2 + 1]);
        rec_sm[(col * L2 + q) * CELL_REC + 8] = (uint32_t)(gprod >> 32);
        rec_sm[(col * L2 + q) * CELL_REC + 9] = mn;
        rec_sm[(col * L2 + q) * CELL_REC + 10] = pl;
        rec_sm[(col * L2 + q) * CELL_REC + 11] = (uint32_t)gprod;
    }
    const size_t rep0 = (size_t)run * NT;
    if (active) {
        const uint32_t* gsp = reinterpret_cast<const uint32_t*>(in.spins + rep0 * N);
        for (int w = j; w < NT * NW; w += TPI) {
            const int buf = w / NW, g = w - buf * NW;
            const int cell = g >> 1, u = g & 1, r = cell / L, c = cell - r * L;
            sw[buf * NWP + ((r + c + u) & 1) * L2 + cell] = gsp[w];
        }
        for (int t = j; t < NT; t += TPI) {
            const uint8_t b = in.perm[rep0 + t];
            Es[t] = in.E[rep0 + t];
            perm[t] = b;
            inv[b] = (uint8_t)t;
            macc[t] = 0u;
            xacc[t] = 0u;
            if (walk) {
                reinterpret_cast<uint32_t*>(ib + lay.whot)[t] = 0u;
                reinterpret_cast<uint32_t*>(ib + lay.wtrips)[t] = 0u;
                (ib + lay.wstate)[t] = in.wstate[rep0 + t];
            }
        }
        if (j == 0) {
            misc[0] = in.best[run];
            misc[1] = in.first[run];
        }
    }
    const int lane = tid & 31;
    const unsigned tmask = G >= 32 ? FULL : (((1u << G) - 1u) << (lane & ~(G - 1)));
    // read through a warp reduction: the keys (and every Philox round key and
    // per-sweep product derived from them) are then warp-uniform values
    const uint32_t k0 = __reduce_or_sync(FULL, in.seed), k1 = __reduce_or_sync(FULL, in.uid);
    const uint32_t runbits = (uint32_t)run << 16;
    const int prep_warp_j0 = TPI >= 32 ? TPI - 32 : 0;
    // a run whose threads start on a warp boundary passes its exchange chain
    // with its first warp; otherwise one thread does
    const bool warp_pass = TPI >= 32 && ((item * TPI) & 31) == 0;
    auto exch = [&](uint32_t sw_) {
        return (NT > 1) && ((mode == 1) || (xevery > 0 && (sw_ % (uint32_t)xevery) == 0u));
    };
    const int n_iter = (mode == 0) ? nsweeps : 1;
    const uint32_t s_first = (mode == 0) ? sweep0 + 1u : sweep0;
    __syncthreads();                            // tables staged before the first exchange preparation
    if (n_iter > 0 && exch(s_first) && active && j >= prep_warp_j0)
        exchange_prepare(in, thr_sm, j - prep_warp_j0, s_first, runbits, k0, k1, NT, ccrit + (s_first & 1u) * NT);
    __syncthreads();

    for (int it = 0; it < n_iter; ++it) {
        const uint32_t s = s_first + (uint32_t)it;
        const bool do_x = exch(s);
        if (mode == 0 && active) {
            const PhiloxSweep ps = philox_sweep_pre(s, k0, k1);
            for (int b = team; b < NT; b += NTEAM) {
                const int t = PT_IDX((int)inv[b], NT, 2u);
                uint32_t* bw = sw + b * NWP;
                const uint32_t* th = thr_sm + t * KTI;
                const uint32_t c1 = runbits | (uint32_t)t;
                int dk = 0, pc = 0;
#pragma unroll
                for (int col = 0; col < 2; ++col) {
                    for (int q = tl; q < L2; q += G) {
                        const uint32_t* rec = rec_sm + (col * L2 + q) * CELL_REC;
                        // group product high half, minus word, plus word, group product low half
                        const uint4 meta = *reinterpret_cast<const uint4*>(rec + 8);
                        const uint4 rn = philox_group_prod(ps, c1, meta.x, meta.w, k0, k1);
                        sm_word(rec, meta, bw, col, L2, q, rn, th, KTI, dk, pc);
                    }
                    __syncwarp(tmask);                  // colour 0 of this buffer done by the whole team
                }
                for (int o = G >> 1; o > 0; o >>= 1) {
                    dk += __shfl_xor_sync(tmask, dk, o);
                    pc += __shfl_xor_sync(tmask, pc, o);
                }
                if (tl == 0) {
                    Es[t] += 2 * dk;
                    macc[t] += (uint32_t)(-pc >> 1);
                }
            }
        }
        __syncthreads();
        if (active && (warp_pass ? j < 32 : j == 0)) {
            int m;
            if (do_x) {
                m = warp_pass ? exchange_chain_warp<true>(Es, perm, inv, xacc, ccrit + (s & 1u) * NT, NT, j)
                              : exchange_chain<true>(Es, perm, inv, xacc, ccrit + (s & 1u) * NT, NT);
                if (WALK && j == 0)
                    walk_update(perm, reinterpret_cast<uint32_t*>(ib + lay.whot),
                                reinterpret_cast<uint32_t*>(ib + lay.wtrips), ib + lay.wstate, NT);
            } else if (warp_pass) {
                m = slot_min_warp(Es, NT, j);
            } else {
                m = Es[0];
                for (int p = 1; p < NT; ++p) m = min(m, Es[p]);
            }
            if (j == 0 && mode == 0 && m < misc[0]) {
                misc[0] = m;
                misc[1] = (int32_t)s;
            }
        }
        if (it + 1 < n_iter && exch(s + 1u) && active && j >= prep_warp_j0)
            exchange_prepare(in, thr_sm, j - prep_warp_j0, s + 1u, runbits, k0, k1, NT,
                             ccrit + ((s + 1u) & 1u) * NT);
        __syncthreads();
    }

    // ---- write the state back
    if (active) {
        uint32_t* gsp = reinterpret_cast<uint32_t*>(in.spins + rep0 * N);
        for (int w = j; w < NT * NW; w += TPI) {
            const int buf = w / NW, g = w - buf * NW;
            const int cell = g >> 1, u = g & 1, r = cell / L, c = cell - r * L;
            gsp[w] = sw[buf * NWP + ((r + c + u) & 1) * L2 + cell];
        }
        for (int t = j; t < NT; t += TPI) {
            in.E[rep0 + t] = Es[t];
            in.perm[rep0 + t] = perm[t];
            in.macc[rep0 + t] += macc[t];
            if (t < NT - 1) in.xacc[(size_t)run * (NT > 1 ? NT - 1 : 1) + t] += xacc[t];
            if (walk) {
                in.whot[rep0 + t] += reinterpret_cast<const uint32_t*>(ib + lay.whot)[t];
                in.wtrips[rep0 + t] += reinterpret_cast<const uint32_t*>(ib + lay.wtrips)[t];
                in.wstate[rep0 + t] = (ib + lay.wstate)[t];
            }
        }
        if (j == 0) {
            in.best[run] = misc[0];
            in.first[run] = misc[1];
        }
    }
    __syncthreads();
}

// SLOT_MAJOR selects the mapping of every bundle of the launch, WALK whether
// the launch tracks the temperature random walk of every copy (separate
// instantiations, so each keeps its own register allocation and the untracked
// kernels carry no walk code).  Both slot-major kernels are bounded to 72
// registers (as if for 896 threads), which keeps 7 CTAs of 128 threads per SM;
// the host still caps slot-major CTAs at 768 threads.
template <bool SLOT_MAJOR, bool WALK, int LT = 0>
__global__ void __launch_bounds__(SLOT_MAJOR ? 896 : MAX_THREADS)
pt_sweep_kernel(const InstDesc* __restrict__ insts, const Bundle* __restrict__ bundles,
                int nbundles, uint32_t sweep0, int nsweeps, int xevery, int mode,
                int* __restrict__ queue)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_next;
    int b = blockIdx.x;
    if (queue) {
        if (threadIdx.x == 0) s_next = atomicAdd(queue, 1);
        __syncthreads();
        b = s_next;
    }
    while (b < nbundles) {
        const Bundle bd = bundles[b];
        if (SLOT_MAJOR)
            process_bundle_sm<WALK, LT>(insts, bd, sweep0, nsweeps, xevery, mode, smem);
        else
            process_bundle<WALK>(insts, bd, sweep0, nsweeps, xevery, mode, smem);
        if (!queue) break;
        if (threadIdx.x == 0) s_next = atomicAdd(queue, 1);
        __syncthreads();
        b = s_next;
        __syncthreads();
    }
}

// Initial spins from the kind-2 stream (counter (0, run << 16 | slot, group, 2)),
// identity slot map, zero counters.  One block per (instance, run).
__global__ void pt_init_kernel(const InstDesc* __restrict__ insts, const int2* __restrict__ items,
                               int draw)
{
    const int2 it = items[blockIdx.x];
    const InstDesc& in = insts[it.x];
    const int run = it.y, NT = in.NT, NW = 2 * in.L * in.L;
    const size_t rep0 = (size_t)run * NT;
    if (draw) {
        uint32_t* gsp = reinterpret_cast<uint32_t*>(in.spins + rep0 * 8 * in.L * in.L);
        for (int w = threadIdx.x; w < NT * NW; w += blockDim.x) {
            const int slot = w / NW, g = w - slot * NW;
            const uint4 r = philox10(0u, ((uint32_t)run << 16) | (uint32_t)slot, (uint32_t)g, 2u,
                                     in.seed, in.uid);
            gsp[w] = ((r.x >> 31) ? 0x000000FFu : 0x00000001u) |
                     ((r.y >> 31) ? 0x0000FF00u : 0x00000100u) |
                     ((r.z >> 31) ? 0x00FF0000u : 0x00010000u) |
                     ((r.w >> 31) ? 0xFF000000u : 0x01000000u);
        }
    }
    for (int t = threadIdx.x; t < NT; t += blockDim.x) {
        in.perm[rep0 + t] = (uint8_t)t;
        in.macc[rep0 + t] = 0ull;
        if (t < NT - 1) in.xacc[(size_t)run * (NT - 1) + t] = 0ull;
    }
}

// Full energies of every slot (Eq. 1 summed over the colour-0 endpoint of each
// coupler), best = min over slots, first = `first_value`.  One block per
// (instance, run), one warp per slot.
__global__ void pt_energy_kernel(const InstDesc* __restrict__ insts, const int2* __restrict__ items,
                                 int32_t first_value)
{
    const int2 it = items[blockIdx.x];
    const InstDesc& in = insts[it.x];
    const int run = it.y, NT = in.NT, L = in.L, L2 = L * L;
    const size_t rep0 = (size_t)run * NT;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    __shared__ int s_min;
    if (threadIdx.x == 0) s_min = INT32_MAX;
    __syncthreads();
    for (int t = warp; t < NT; t += nwarps) {
        const int buf = PT_IDX((int)in.perm[rep0 + t], NT, 7u);
        const uint32_t* w = reinterpret_cast<const uint32_t*>(in.spins + (rep0 + buf) * 8 * L2);
        int acc = 0;
        for (int q = lane; q < L2; q += 32) {
            const int r = q / L, c = q - r * L, u = (r + c) & 1;      // colour-0 group of cell q
            const uint32_t* jw = in.jw + (q * 2 + 0) * 8;
            const uint32_t own = w[2 * q + u];
            const int opp = (int)w[2 * q + (1 - u)];
            const uint32_t mw = w[2 * in.nbr[(q * 2) * 2 + 0] + u];
            const uint32_t pw = w[2 * in.nbr[(q * 2) * 2 + 1] + u];
            const int x01 = (int)__byte_perm(mw, pw, 0x5140), x23 = (int)__byte_perm(mw, pw, 0x7362);
            const int h0 = __dp4a((int)jw[0], opp, __dp4a((int)jw[4], x01, 0));
            const int h1 = __dp4a((int)jw[1], opp, __dp4a((int)jw[5], x01, 0));
            const int h2 = __dp4a((int)jw[2], opp, __dp4a((int)jw[6], x23, 0));
            const int h3 = __dp4a((int)jw[3], opp, __dp4a((int)jw[7], x23, 0));
            acc -= (int)(int8_t)own * h0 + (int)(int8_t)(own >> 8) * h1 +
                   (int)(int8_t)(own >> 16) * h2 + (int)(int8_t)(own >> 24) * h3;
        }
        const int e = __reduce_add_sync(FULL, acc);
        if (lane == 0) {
            in.E[rep0 + t] = e;
            atomicMin(&s_min, e);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        in.best[run] = s_min;
        in.first[run] = first_value;
    }
}

// Time to solution per instance: target = explicit or min best, hit if
// best <= target and first <= horizon, lower median (rank ceil(R/2)) of hit
// sweeps with misses as +inf, horizon + 1 when unsolved.  One block per instance.
__global__ void pt_tts_kernel(const InstDesc* __restrict__ insts, int32_t target, int32_t horizon,
                              int32_t* __restrict__ out, const int32_t* __restrict__ targets)
{
    const InstDesc& in = insts[blockIdx.x];
    if (targets) target = targets[blockIdx.x];
#ifdef PT_DEBUG
    const int R = in.R > 1024 ? (atomicCAS(&g_pt_debug_code, 0u, 6u), 1024) : in.R;
#else
    const int R = in.R;
#endif
    __shared__ long long v[1024];
    __shared__ int s_min, s_hits;
    __shared__ long long s_med;
    const long long INF = 0x7FFFFFFFFFFFFFFFll;
    if (threadIdx.x == 0) {
        s_min = INT32_MAX;
        s_hits = 0;
        s_med = INF;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < R; r += blockDim.x) atomicMin(&s_min, in.best[r]);
    __syncthreads();
    const int T = (target == INT32_MAX) ? s_min : target;
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
        const bool hit = in.best[r] <= T && in.first[r] <= horizon;
        v[r] = hit ? (long long)in.first[r] : INF;
        if (hit) atomicAdd(&s_hits, 1);
    }
    __syncthreads();
    const int m = (R + 1) / 2 - 1;
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
        int rank = 0;
        for (int x = 0; x < R; ++x) rank += (v[x] < v[r]) || (v[x] == v[r] && x < r);
        if (rank == m) s_med = v[r];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        out[blockIdx.x * 3 + 0] = (s_med == INF) ? horizon + 1 : (int32_t)s_med;
        out[blockIdx.x * 3 + 1] = s_hits;
        out[blockIdx.x * 3 + 2] = T;
    }
}

// Hamming distances between n sampled configurations of instance 0, sample
// k being slot slot[k] of run run[k]: dist[k][k2] (block k, thread k2).
// Spins are +-1 bytes, so two differ exactly when their XOR is 0xFE (7 bits).
__global__ void pt_hamming_kernel(const InstDesc* __restrict__ insts, int n, const int32_t* __restrict__ run,
                                  const int32_t* __restrict__ slot, int32_t* __restrict__ dist)
{
    const InstDesc& in = insts[0];
    const int NT = in.NT, NW = 2 * in.L * in.L;
    auto conf = [&](int k) {
        const size_t rep = (size_t)run[k] * NT;
        return reinterpret_cast<const uint32_t*>(in.spins + (rep + in.perm[rep + slot[k]]) * 4 * NW);
    };
    const int k = blockIdx.x;
    const uint32_t* a = conf(k);
    for (int k2 = threadIdx.x; k2 < n; k2 += blockDim.x) {
        const uint32_t* b = conf(k2);
        int bits = 0;
        for (int w = 0; w < NW; ++w) bits += __popc(a[w] ^ b[w]);
        dist[(size_t)k * n + k2] = bits / 7;
    }
}

}  // namespace

#ifdef PT_DEBUG
namespace {
std::atomic<unsigned> g_debug_sticky{0};
}
bool debug_build() { return true; }
cudaError_t debug_check(cudaStream_t st, const char* what)
{
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess || cap != cudaStreamCaptureStatusNone) return e;   // checked after the graph replay
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    unsigned code = 0;
    if ((e = cudaMemcpyFromSymbol(&code, g_pt_debug_code, sizeof(code))) != cudaSuccess) return e;
    if (code) {
        const unsigned zero = 0;
        if ((e = cudaMemcpyToSymbol(g_pt_debug_code, &zero, sizeof(zero))) != cudaSuccess) return e;
        unsigned expect = 0;
        g_debug_sticky.compare_exchange_strong(expect, code);
        std::fprintf(stderr, "PT_DEBUG: bounds check %u failed in %s\n", code, what);
    }
    return cudaSuccess;
}
unsigned debug_take() { return g_debug_sticky.exchange(0u); }
#define DBG(e, st, what) ((e) == cudaSuccess ? debug_check((st), (what)) : (e))
#else
bool debug_build() { return false; }
cudaError_t debug_check(cudaStream_t, const char*) { return cudaSuccess; }
unsigned debug_take() { return 0u; }
#define DBG(e, st, what) (e)
#endif

cudaError_t sweep_smem_capacity(int* bytes)
{
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    size_t stat = 0;
    const void* ks[12] = {(const void*)pt_sweep_kernel<false, false>, (const void*)pt_sweep_kernel<true, false>,
                          (const void*)pt_sweep_kernel<false, true>, (const void*)pt_sweep_kernel<true, true>,
                          (const void*)pt_sweep_kernel<true, false, 4>, (const void*)pt_sweep_kernel<true, false, 8>,
                          (const void*)pt_sweep_kernel<true, false, 12>, (const void*)pt_sweep_kernel<true, false, 16>,
                          (const void*)pt_sweep_kernel<true, true, 4>, (const void*)pt_sweep_kernel<true, true, 8>,
                          (const void*)pt_sweep_kernel<true, true, 12>, (const void*)pt_sweep_kernel<true, true, 16>};
    for (const void* k : ks) {
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, k);
        if (e != cudaSuccess) return e;
        stat = fa.sharedSizeBytes > stat ? fa.sharedSizeBytes : stat;
    }
    *bytes = optin - (int)stat;
    return cudaSuccess;
}

cudaError_t sweep_occupancy(int block, int smem_bytes, int* blocks_per_sm, bool slot_major, bool walk)
{
    const void* k = slot_major ? (walk ? (const void*)pt_sweep_kernel<true, true> : (const void*)pt_sweep_kernel<true, false>)
                               : (walk ? (const void*)pt_sweep_kernel<false, true> : (const void*)pt_sweep_kernel<false, false>);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, block, smem_bytes);
}

cudaError_t set_sweep_smem_limit(int bytes)
{
    const void* ks[12] = {(const void*)pt_sweep_kernel<false, false>, (const void*)pt_sweep_kernel<true, false>,
                          (const void*)pt_sweep_kernel<false, true>, (const void*)pt_sweep_kernel<true, true>,
                          (const void*)pt_sweep_kernel<true, false, 4>, (const void*)pt_sweep_kernel<true, false, 8>,
                          (const void*)pt_sweep_kernel<true, false, 12>, (const void*)pt_sweep_kernel<true, false, 16>,
                          (const void*)pt_sweep_kernel<true, true, 4>, (const void*)pt_sweep_kernel<true, true, 8>,
                          (const void*)pt_sweep_kernel<true, true, 12>, (const void*)pt_sweep_kernel<true, true, 16>};
    for (const void* k : ks) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_init(const InstDesc* insts, const int2* items, int nitems, bool draw,
                        cudaStream_t st)
{
    if (nitems <= 0) return cudaSuccess;
    pt_init_kernel<<<nitems, 256, 0, st>>>(insts, items, draw ? 1 : 0);
    return DBG(cudaGetLastError(), st, "init kernel");
}

cudaError_t launch_energy(const InstDesc* insts, const int2* items, int nitems, int32_t first_value,
                          cudaStream_t st)
{
    if (nitems <= 0) return cudaSuccess;
    pt_energy_kernel<<<nitems, 256, 0, st>>>(insts, items, first_value);
    return DBG(cudaGetLastError(), st, "energy kernel");
}

cudaError_t launch_sweeps(const InstDesc* insts, const Bundle* bundles, int nbundles, int grid,
                          int block, int smem_bytes, uint32_t sweep0, int nsweeps, int xevery,
                          int mode, int* queue, cudaStream_t st, bool slot_major, bool walk, int L)
{
    if (nbundles <= 0) return cudaSuccess;
#define PT_SM_LAUNCH(W, LT)                                                                                   \
    pt_sweep_kernel<true, W, LT><<<grid, block, smem_bytes, st>>>(insts, bundles, nbundles, sweep0, nsweeps, \
                                                                  xevery, mode, queue)
#define PT_SM_LAUNCH_L(W)                                                                                     \
    do {                                                                                                      \
        if (L == 4) PT_SM_LAUNCH(W, 4);                                                                       \
        else if (L == 8) PT_SM_LAUNCH(W, 8);                                                                  \
        else if (L == 12) PT_SM_LAUNCH(W, 12);                                                                \
        else if (L == 16) PT_SM_LAUNCH(W, 16);                                                                \
        else PT_SM_LAUNCH(W, 0);                                                                              \
    } while (0)
    if (slot_major && walk)
        PT_SM_LAUNCH_L(true);
    else if (slot_major)
        PT_SM_LAUNCH_L(false);
#undef PT_SM_LAUNCH_L
#undef PT_SM_LAUNCH
    else if (walk)
        pt_sweep_kernel<false, true><<<grid, block, smem_bytes, st>>>(insts, bundles, nbundles, sweep0, nsweeps,
                                                                      xevery, mode, queue);
    else
        pt_sweep_kernel<false, false><<<grid, block, smem_bytes, st>>>(insts, bundles, nbundles, sweep0, nsweeps,
                                                                       xevery, mode, queue);
    return DBG(cudaGetLastError(), st, "sweep kernel");
}

cudaError_t launch_hamming(const InstDesc* insts, int n, const int32_t* run, const int32_t* slot, int32_t* dist,
                           cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    pt_hamming_kernel<<<n, 256, 0, st>>>(insts, n, run, slot, dist);
    return DBG(cudaGetLastError(), st, "hamming kernel");
}

cudaError_t launch_tts(const InstDesc* insts, int ninst, int32_t target, int32_t horizon,
                       int32_t* out, cudaStream_t st, const int32_t* targets)
{
    if (ninst <= 0) return cudaSuccess;
    pt_tts_kernel<<<ninst, 256, 0, st>>>(insts, target, horizon, out, targets);
    return DBG(cudaGetLastError(), st, "TTS kernel");
}

}  // namespace ptg
