// pt_internal.h -- device data layout shared by the kernels and the host runtime
// of the GB300 PT engine (library-private; the public ABI is include/pt.h).
#pragma once
#include <cstdint>
#ifndef __CUDACC__
#define __host__
#define __device__
#endif

namespace ptg {

// Metropolis table rows per temperature slot: k = 0 .. kt-1 where kt - 1 is
// the largest local-field magnitude K = max_i sum_j |J_ij| an instance can
// produce.  Couplers in {+-1, +-2, +-3} give K <= 18 (the default row count);
// planted instances with summed loop weights need more, up to KT_MAX - 1.
constexpr int KT_DEFAULT = 19;
constexpr int KT_MAX = 128;
constexpr int J_ABS_MAX = 127;     // couplers are int8
constexpr int MAX_TEMPS = 64;
constexpr int MAX_L = 16;
constexpr int MAX_THREADS = 1024;
// CTA size limit of the slot-major sweep kernel: its register budget (up to
// 80 per thread) fits 768 threads per CTA.
constexpr int MAX_THREADS_SM = 768;

// Per instance.  All pointers are device pointers.
//
// Couplers are repacked per (cell, colour): the cell's group of 4 spins of
// that colour (orientation u = (r + c + colour) & 1) needs
//   jin[k]  bytes k' = 0..3: -J to the 4 opposite-orientation spins of the cell
//   jud[k]  -J to the inter-cell neighbours of spin k: spin 0/2 in bytes 0,1,
//           spin 1/3 in bytes 2,3 (minus-side neighbour first)
// stored as jw[(cell * 2 + colour) * 8 + {0..3 jin, 4..7 jud}].  The negation
// makes dp4a produce -h_i directly.  nbr[(cell * 2 + colour) * 2 + {0,1}] is the
// minus/plus neighbour cell of that group (the cell itself where absent; its
// couplers are 0 there).
struct InstDesc {
    int32_t L, NT, R, n_xpairs;
    uint32_t seed, uid;
    int32_t kt;               // Metropolis table rows per slot (> every spin's sum of |J|)
    const uint32_t* jw;
    const int16_t* nbr;
    const uint32_t* thr;      // [NT][kt]; entry 0 = 0xFFFFFFFF (unused: k <= 0 always accepts)
    const int32_t* xoff;      // [NT]  pair p owns xthr[xoff[p] .. xoff[p+1]-1], h = 1..H_p
    const uint32_t* xthr;
    const float* xhint;       // [NT-1] ln2 / (2 dbeta_p): start point of the exact table search
    int8_t* spins;            // [R][NT][N] by configuration buffer, natural spin order
    int32_t* E;               // [R][NT] by slot
    uint8_t* perm;            // [R][NT] slot -> buffer
    int32_t* best;            // [R]
    int32_t* first;           // [R]
    unsigned long long* macc; // [R][NT] accepted flips per slot
    unsigned long long* xacc; // [R][max(NT-1,1)] accepted swaps per pair
    // temperature random walk of each system copy (= configuration buffer);
    // all three NULL when the walk is not tracked
    unsigned long long* whot = nullptr;   // [R][NT] exchange passes spent in the hot half
    unsigned long long* wtrips = nullptr; // [R][NT] completed cold -> hot -> cold round trips
    uint8_t* wstate = nullptr;            // [R][NT] 0 none, 1 coldest slot seen, 2 then hottest
};

// One CTA work unit: `nitems` consecutive runs of one instance.
//   team == 0 (cell-major): sp * L^2 threads per run; a thread owns one cell
//              and every sp-th temperature slot.
//   team  > 0 (slot-major): sp teams of `team` lanes (a power of two <= 32)
//              per run; a team owns every sp-th slot, its lanes split the cells.
struct Bundle {
    int32_t inst, run0, nitems, sp, team;
};

__host__ __device__ inline int threads_per_run(int L, const Bundle& b)
{
    return b.team > 0 ? b.sp * b.team : b.sp * L * L;
}

// Shared-memory layout of one bundle: the Metropolis table of the instance,
// then per item (run): spins [NT][N] (colour-major words per buffer, plus
// `pad` words per buffer in the slot-major mapping), E by slot, exchange
// critical h by pair (two sweeps), flip / swap counters, perm (slot ->
// buffer), its inverse (buffer -> slot, slot-major mapping), best/first.
struct ItemLayout {
    int64_t spins, E, ccrit, macc, xacc, perm, inv, whot, wtrips, wstate, misc, bytes;
};

__host__ __device__ inline int64_t pad16(int64_t x) { return (x + 15) & ~15LL; }

__host__ __device__ inline ItemLayout item_layout(int L, int NT, int pad = 0, bool walk = false)
{
    ItemLayout o;
    const int64_t N = 8LL * L * L;
    o.spins = 0;
    o.E = pad16((int64_t)NT * (N + 4LL * pad));
    o.ccrit = o.E + 4LL * NT;
    o.macc = o.ccrit + 8LL * NT;
    o.xacc = o.macc + 4LL * NT;
    o.perm = o.xacc + 4LL * NT;
    o.inv = o.perm + NT;
    int64_t end = o.inv + NT;
    if (walk) {                       // per-copy walk counters for this launch, and walk states
        o.whot = (end + 3) & ~3LL;
        o.wtrips = o.whot + 4LL * NT;
        o.wstate = o.wtrips + 4LL * NT;
        end = o.wstate + NT;
    } else {
        o.whot = o.wtrips = o.wstate = end;
    }
    o.misc = pad16(end);
    o.bytes = o.misc + 16;
    return o;
}

// Slot-major mapping: padding words per spin buffer so that the buffer
// stride is congruent to the team width modulo the 32 shared-memory banks.
// Teams of one warp own consecutive buffers and their lanes read consecutive
// words, so the spin words a warp reads at once fall into distinct banks.
__host__ __device__ inline int sm_pad(int L, int team)
{
    const int NW = 2 * L * L;
    return ((team & 31) - (NW & 31) + 64) & 31;
}

// Instance tables staged per bundle: thr [NT][kt], then exchange offsets [NT]
// and search hints [NT].
__host__ __device__ inline int64_t table_bytes(int NT, int kt) { return pad16(4LL * NT * kt + 8LL * NT); }

// Sets the message pt_last_error(NULL) returns (defined with the C ABI).
void set_global_error(const char* msg);

// Slot-major mapping only: one 12-word record per (colour, cell), colour-major:
// in-cell couplers (4 words), inter-cell couplers (4 words), then one 16-byte
// word group read by a single load with no unpacking: the high half of the
// Philox round-0 product M1 * (group index), the minus- and plus-neighbour
// spin word, the low half of that product.  The 48-byte stride puts the
// records a team reads at once into distinct banks.
constexpr int CELL_REC = 12;
__host__ __device__ inline int64_t cell_table_bytes(int L) { return 4LL * CELL_REC * 2 * L * L; }

inline int64_t bundle_smem_bytes(int L, int NT, int nitems, int team = 0, bool walk = false, int kt = KT_DEFAULT)
{
    if (team > 0)
        return table_bytes(NT, kt) + cell_table_bytes(L) +
               (int64_t)nitems * item_layout(L, NT, sm_pad(L, team), walk).bytes;
    return table_bytes(NT, kt) + (int64_t)nitems * item_layout(L, NT, 0, walk).bytes;
}

}  // namespace ptg
