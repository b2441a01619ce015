/*
 * pt_oracle.c -- plain, slow, single-threaded CPU oracle.
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline leg may load this library.  It shares no code, header, table or
 * constant generator with the CUDA path: everything below is written out again
 * from the definitions it cites.
 *
 * What it computes (arXiv:1605.03607, "Practical engineering of hard
 * spin-glass instances"):
 *   - the Ising cost H = sum_<ij> J_ij s_i s_j over the couplers of the
 *     Chimera graph, minimised over s_i = +-1 (Eq. 1; graph of Appendix A,
 *     Fig. 8: L x L unit cells of K_{4,4});
 *   - parallel tempering (Sec. II): N_T copies at inverse temperatures
 *     beta_0 > beta_1 > ... (slot 0 coldest), independent Metropolis sweeps,
 *     then a temperature-exchange sweep over neighbouring pairs with the
 *     detailed-balance acceptance min(1, exp((beta_p - beta_{p+1})(E_p - E_{p+1})));
 *     a sweep is a full-lattice Metropolis sweep (Sec. III.B, EMCS definition);
 *   - the hardness figure of merit "time to solution" (Sec. II) in the form
 *     used here: the lower median over independent PT runs of the first sweep
 *     at which a run reaches the target energy;
 *   - one step of random adaptive optimisation (Algorithm 1): perturb one
 *     coupler, re-measure TTS, keep the change if TTS increased, otherwise keep
 *     it with probability exp(-beta_RAO |dTTS|) (greedy when beta_RAO = inf).
 *   - the temperature random walk of every system copy (Sec. III.B): passes
 *     spent in the hot half of the ladder and completed round trips;
 *   - planted-solution instances built from frustrated loops and one step of
 *     loop adaptive optimisation (Sec. IV, Algorithm 2), with the TTS taken
 *     against the known ground-state energy.
 *
 * Readings where the paper is silent (all fixed identically on both sides):
 *   - spin index i = 8*(r*L + c) + 4*u + k (u = 0 vertical, u = 1 horizontal);
 *     edge order: intra-cell (cell-major, k, k'), then vertical inter-cell
 *     (r, c, k), then horizontal inter-cell (r, c, k);
 *   - sweep = colour 0 spins then colour 1 spins, colour (r + c + u) mod 2
 *     (the two sides of the bipartite graph), each colour in index order;
 *   - Metropolis on the integer k = -s_i h_i (dE = 2k): accept if k <= 0,
 *     else if u < thr[slot][k] with thr = floor(exp(-2 k beta) 2^32) built in
 *     FP64 (acceptance exact to 2^-32);
 *   - exchange after every `exchange_every`-th sweep, pairs p = 0..N_T-2 in
 *     ascending order (chained swaps allowed); energies of one instance differ
 *     by even numbers, d = E_{p+1} - E_p = 2h: accept if h <= 0, else if
 *     h <= H_p and u < xthr[p][h] = floor(exp(-2 h (beta_p - beta_{p+1})) 2^32);
 *     configurations are swapped whole (this oracle keeps no permutation);
 *   - temperature random walk: a system copy is identified by the slot its
 *     configuration started in; its hot-half time is counted in exchange
 *     passes, the hot half being the N_T/2 highest temperatures;
 *   - random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11),
 *     key = (seed, uid), counter (sweep, run<<16 | slot, group, kind) with
 *     kind 0 Metropolis (group = i>>2, word i&3), 1 exchange (group = p>>2,
 *     word p&3, slot field 0), 2 initial spins (sweep 0; s = -1 if the word's
 *     top bit is set), 3 engineering draws (counter (step, proposal, 0, 3)).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define OR_KMAX_LIMIT 127    /* largest |h_i| an instance may have (sum of |J| over a spin's couplers) */
#define OR_HMAX (1 << 22)    /* cap on the exchange table length per pair */

/* ------------------------------------------------------------------ */
/* Philox4x32-10, written from its published definition (SC'11).       */
/* ------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {                 /* Weyl key schedule between rounds */
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static uint32_t draw(uint32_t seed, uint32_t uid, uint32_t c0, uint32_t c1,
                     uint32_t c2, uint32_t c3, int word)
{
    uint32_t ctr[4] = {c0, c1, c2, c3}, key[2] = {seed, uid}, out[4];
    or_philox4x32_10(ctr, key, out);
    return out[word];
}

/* ------------------------------------------------------------------ */
/* Chimera graph (Appendix A, Fig. 8).                                 */
/* ------------------------------------------------------------------ */
static int spin_index(int L, int r, int c, int u, int k) { return 8 * (r * L + c) + 4 * u + k; }

int or_chimera_n_edges(int L) { return 16 * L * L + 8 * L * (L - 1); }

/* Fills ei/ej (capacity or_chimera_n_edges(L)); returns the edge count. */
int or_chimera_edges(int L, int32_t *ei, int32_t *ej)
{
    int e = 0;
    for (int r = 0; r < L; ++r)                       /* intra-cell K_{4,4} */
        for (int c = 0; c < L; ++c)
            for (int k = 0; k < 4; ++k)
                for (int kp = 0; kp < 4; ++kp) {
                    ei[e] = spin_index(L, r, c, 0, k);
                    ej[e] = spin_index(L, r, c, 1, kp);
                    ++e;
                }
    for (int r = 0; r + 1 < L; ++r)                   /* vertical: (r,c,0,k)-(r+1,c,0,k) */
        for (int c = 0; c < L; ++c)
            for (int k = 0; k < 4; ++k) {
                ei[e] = spin_index(L, r, c, 0, k);
                ej[e] = spin_index(L, r + 1, c, 0, k);
                ++e;
            }
    for (int r = 0; r < L; ++r)                       /* horizontal: (r,c,1,k)-(r,c+1,1,k) */
        for (int c = 0; c + 1 < L; ++c)
            for (int k = 0; k < 4; ++k) {
                ei[e] = spin_index(L, r, c, 1, k);
                ej[e] = spin_index(L, r, c + 1, 1, k);
                ++e;
            }
    return e;
}

int or_spin_colour(int L, int i)
{
    int cell = i >> 3, r = cell / L, c = cell % L, u = (i >> 2) & 1;
    return (r + c + u) & 1;
}

/* Eq. 1: H = sum over couplers of J_e s_i s_j. */
int32_t or_energy(int L, const int8_t *J, const int8_t *s)
{
    int E = or_chimera_n_edges(L);
    int32_t *ei = malloc(sizeof(int32_t) * E), *ej = malloc(sizeof(int32_t) * E);
    or_chimera_edges(L, ei, ej);
    int64_t H = 0;
    for (int e = 0; e < E; ++e) H += (int64_t)J[e] * s[ei[e]] * s[ej[e]];
    free(ei); free(ej);
    return (int32_t)H;
}

/* Neighbour lists: for spin i, up to 6 (neighbour, J) pairs. */
typedef struct { int n; int32_t nb[6]; int8_t Jn[6]; } nbr_list;

static nbr_list *build_neighbours(int L, const int8_t *J)
{
    int N = 8 * L * L, E = or_chimera_n_edges(L);
    int32_t *ei = malloc(sizeof(int32_t) * E), *ej = malloc(sizeof(int32_t) * E);
    or_chimera_edges(L, ei, ej);
    nbr_list *nl = calloc((size_t)N, sizeof(nbr_list));
    for (int e = 0; e < E; ++e) {
        nbr_list *a = &nl[ei[e]], *b = &nl[ej[e]];
        a->nb[a->n] = ej[e]; a->Jn[a->n] = J[e]; a->n++;
        b->nb[b->n] = ei[e]; b->Jn[b->n] = J[e]; b->n++;
    }
    free(ei); free(ej);
    return nl;
}

/* ------------------------------------------------------------------ */
/* Acceptance tables, FP64 on the host.                                */
/* ------------------------------------------------------------------ */
static uint32_t prob_to_u32(double p)
{
    double x = floor(ldexp(p, 32));
    if (x >= 4294967295.0) return 0xFFFFFFFFu;
    if (x <= 0.0) return 0u;
    return (uint32_t)x;
}

/* thr[t*(kmax+1) + k] = floor(exp(-2 k beta_t) 2^32) for k = 1..kmax; entry 0 unused (0). */
void or_metropolis_thresholds(int n_temps, const double *betas, int kmax, uint32_t *thr)
{
    for (int t = 0; t < n_temps; ++t) {
        thr[t * (kmax + 1)] = 0;
        for (int k = 1; k <= kmax; ++k)
            thr[t * (kmax + 1) + k] = prob_to_u32(exp(-2.0 * (double)k * betas[t]));
    }
}

/* The largest local-field magnitude the couplers allow: max over spins of
 * the sum of |J| over the spin's couplers (k = -s_i h_i never exceeds it). */
int or_coupler_kmax(int L, const int8_t *J)
{
    int N = 8 * L * L, E = or_chimera_n_edges(L);
    int32_t *ei = malloc(sizeof(int32_t) * E), *ej = malloc(sizeof(int32_t) * E);
    int *sum = calloc((size_t)N, sizeof(int));
    or_chimera_edges(L, ei, ej);
    for (int e = 0; e < E; ++e) {
        int a = J[e] < 0 ? -J[e] : J[e];
        sum[ei[e]] += a;
        sum[ej[e]] += a;
    }
    int m = 0;
    for (int i = 0; i < N; ++i) if (sum[i] > m) m = sum[i];
    free(ei); free(ej); free(sum);
    return m;
}

/* Length H_p of pair p's exchange table: the largest h with a nonzero entry. */
static int exchange_len(double dbeta)
{
    int h = 0;
    while (h < OR_HMAX && prob_to_u32(exp(-2.0 * (double)(h + 1) * dbeta)) != 0) ++h;
    return h;
}

/* Ragged exchange tables: pair p owns entries off[p] .. off[p+1]-1 for h = 1..H_p.
 * Returns the total length (needs off of n_temps entries).  table may be NULL
 * to query the size.  Returns -1 if the ladder is not strictly descending. */
int64_t or_exchange_thresholds(int n_temps, const double *betas, int64_t *off, uint32_t *table)
{
    int64_t total = 0;
    for (int p = 0; p + 1 < n_temps; ++p) {
        double dbeta = betas[p] - betas[p + 1];
        if (!(dbeta > 0.0)) return -1;
        int H = exchange_len(dbeta);
        if (off) off[p] = total;
        if (table)
            for (int h = 1; h <= H; ++h)
                table[total + h - 1] = prob_to_u32(exp(-2.0 * (double)h * dbeta));
        total += H;
    }
    if (off && n_temps > 0) off[n_temps - 1] = total;
    return total;
}

/* ------------------------------------------------------------------ */
/* Parallel tempering.                                                  */
/* State arrays (slot order; configurations are swapped physically):   */
/*   spins[(run*NT + slot)*N + i], E[run*NT + slot],                    */
/*   best[run], first[run], macc[run*NT + slot] (accepted flips),       */
/*   xacc[run*(NT-1) + p] (accepted exchanges of pair p).              */
/* ------------------------------------------------------------------ */
void or_pt_init_spins(int L, int n_temps, int n_runs, uint32_t seed, uint32_t uid, int8_t *spins)
{
    int N = 8 * L * L;
    for (int run = 0; run < n_runs; ++run)
        for (int t = 0; t < n_temps; ++t)
            for (int i = 0; i < N; ++i) {
                uint32_t w = draw(seed, uid, 0u, ((uint32_t)run << 16) | (uint32_t)t,
                                  (uint32_t)(i >> 2), 2u, i & 3);
                spins[((size_t)run * n_temps + t) * N + i] = (w >> 31) ? -1 : 1;
            }
}

/* Full energies; best = min over slots of each run, first = 0. */
void or_pt_start(int L, const int8_t *J, int n_temps, int n_runs, const int8_t *spins,
                 int32_t *E, int32_t *best, int32_t *first)
{
    int N = 8 * L * L;
    for (int run = 0; run < n_runs; ++run) {
        int32_t m = INT32_MAX;
        for (int t = 0; t < n_temps; ++t) {
            int32_t e = or_energy(L, J, spins + ((size_t)run * n_temps + t) * N);
            E[run * n_temps + t] = e;
            if (e < m) m = e;
        }
        best[run] = m;
        first[run] = 0;
    }
}

typedef struct {
    int L, N, NT, R, kmax;
    uint32_t seed, uid;
    nbr_list *nl;
    uint32_t *thr;            /* [NT][kmax + 1] */
    int64_t *xoff;
    uint32_t *xthr;
} pt_ctx;

static int ctx_open(pt_ctx *cx, int L, const int8_t *J, int n_temps, const double *betas,
                    int n_runs, uint32_t seed, uint32_t uid)
{
    cx->L = L; cx->N = 8 * L * L; cx->NT = n_temps; cx->R = n_runs;
    cx->seed = seed; cx->uid = uid;
    cx->nl = build_neighbours(L, J);
    cx->kmax = or_coupler_kmax(L, J);
    cx->thr = malloc(sizeof(uint32_t) * (size_t)n_temps * (cx->kmax + 1));
    or_metropolis_thresholds(n_temps, betas, cx->kmax, cx->thr);
    cx->xoff = malloc(sizeof(int64_t) * (size_t)(n_temps > 0 ? n_temps : 1));
    int64_t tot = or_exchange_thresholds(n_temps, betas, NULL, NULL);
    if (tot < 0) return -1;
    cx->xthr = malloc(sizeof(uint32_t) * (size_t)(tot > 0 ? tot : 1));
    or_exchange_thresholds(n_temps, betas, cx->xoff, cx->xthr);
    return 0;
}

static void ctx_close(pt_ctx *cx)
{
    free(cx->nl); free(cx->thr); free(cx->xoff); free(cx->xthr);
}

/* One full-lattice Metropolis sweep of one copy (colour 0 then colour 1). */
static void metropolis_sweep(const pt_ctx *cx, int run, int slot, uint32_t sweep,
                             int8_t *s, int32_t *E, uint64_t *macc)
{
    const uint32_t *thr = cx->thr + (size_t)slot * (cx->kmax + 1);
    for (int colour = 0; colour < 2; ++colour)
        for (int i = 0; i < cx->N; ++i) {
            if (or_spin_colour(cx->L, i) != colour) continue;
            const nbr_list *nb = &cx->nl[i];
            int h = 0;
            for (int a = 0; a < nb->n; ++a) h += nb->Jn[a] * s[nb->nb[a]];
            int k = -s[i] * h;                         /* dE = 2k */
            uint32_t u = draw(cx->seed, cx->uid, sweep,
                              ((uint32_t)run << 16) | (uint32_t)slot,
                              (uint32_t)(i >> 2), 0u, i & 3);
            int accept = (k <= 0) || (u < thr[k]);
            if (accept) {
                s[i] = (int8_t)-s[i];
                *E += 2 * k;
                *macc += 1;
            }
        }
}

/* Temperature random walk of the copies of one run (Sec. III.B), kept when
 * `copy` is not NULL: copy[t] is the id of the copy (the slot it started in)
 * whose configuration sits in slot t.  After an exchange pass, each copy in
 * the hot half -- the NT/2 highest temperatures, slots NT - NT/2 .. NT-1 --
 * counts one more pass there (the paper's first mixing criterion is the
 * least of these over copies), and the copy in the coldest slot completes a
 * round trip if it reached the hottest slot since it last sat in the coldest
 * one (state 0: neither end seen yet, 1: coldest seen, 2: hottest seen
 * after it). */
typedef struct {
    int32_t *copy;      /* [NT] slot -> copy */
    uint64_t *hot;      /* [NT] by copy */
    uint64_t *trips;    /* [NT] by copy */
    uint8_t *state;     /* [NT] by copy */
} walk_run;

static void walk_after_pass(int NT, const walk_run *w)
{
    for (int t = NT - NT / 2; t < NT; ++t) w->hot[w->copy[t]] += 1;
    int c = w->copy[0];
    if (w->state[c] == 2) w->trips[c] += 1;
    w->state[c] = 1;
    int h = w->copy[NT - 1];
    if (w->state[h] == 1) w->state[h] = 2;
}

/* One exchange sweep of one run: pairs p = 0..NT-2 in ascending order. */
static void exchange_pass(const pt_ctx *cx, int run, uint32_t sweep, int8_t *spins_run,
                          int32_t *E_run, uint64_t *xacc_run, const walk_run *w)
{
    int N = cx->N;
    int8_t *tmp = malloc((size_t)N);
    for (int p = 0; p + 1 < cx->NT; ++p) {
        int32_t d = E_run[p + 1] - E_run[p];          /* always even */
        int32_t h = d / 2;
        uint32_t u = draw(cx->seed, cx->uid, sweep, (uint32_t)run << 16,
                          (uint32_t)(p >> 2), 1u, p & 3);
        int accept;
        if (h <= 0) accept = 1;
        else {
            int64_t H = cx->xoff[p + 1] - cx->xoff[p];
            accept = (h <= H) && (u < cx->xthr[cx->xoff[p] + h - 1]);
        }
        if (accept) {
            memcpy(tmp, spins_run + (size_t)p * N, (size_t)N);
            memcpy(spins_run + (size_t)p * N, spins_run + (size_t)(p + 1) * N, (size_t)N);
            memcpy(spins_run + (size_t)(p + 1) * N, tmp, (size_t)N);
            int32_t e = E_run[p]; E_run[p] = E_run[p + 1]; E_run[p + 1] = e;
            xacc_run[p] += 1;
            if (w) { int32_t c = w->copy[p]; w->copy[p] = w->copy[p + 1]; w->copy[p + 1] = c; }
        }
    }
    free(tmp);
    if (w && cx->NT > 1) walk_after_pass(cx->NT, w);
}

static walk_run walk_of_run(int n_temps, int run, int32_t *copy, uint64_t *hot, uint64_t *trips,
                            uint8_t *state)
{
    walk_run w;
    size_t o = (size_t)run * n_temps;
    w.copy = copy + o; w.hot = hot + o; w.trips = trips + o; w.state = state + o;
    return w;
}

/* Runs sweeps sweep0+1 .. sweep0+n_sweeps in place.  After each sweep s the
 * per-run best energy / first sweep are updated, then, if exchange_every > 0
 * and s % exchange_every == 0, one exchange sweep with counter sweep = s.
 * The walk arrays ([n_runs][n_temps] each) are all NULL or all given. */
int or_pt_sweeps_walk(int L, const int8_t *J, int n_temps, const double *betas, int n_runs,
                      uint32_t seed, uint32_t uid, int8_t *spins, int32_t *E, int32_t *best,
                      int32_t *first, uint64_t *macc, uint64_t *xacc, uint32_t sweep0,
                      int n_sweeps, int exchange_every, int32_t *copy, uint64_t *hot,
                      uint64_t *trips, uint8_t *state)
{
    pt_ctx cx;
    if (ctx_open(&cx, L, J, n_temps, betas, n_runs, seed, uid) != 0) { ctx_close(&cx); return -1; }
    int N = cx.N;
    for (int run = 0; run < n_runs; ++run) {
        int8_t *sr = spins + (size_t)run * n_temps * N;
        int32_t *Er = E + (size_t)run * n_temps;
        walk_run w;
        if (copy) w = walk_of_run(n_temps, run, copy, hot, trips, state);
        for (int step = 1; step <= n_sweeps; ++step) {
            uint32_t s = sweep0 + (uint32_t)step;
            for (int t = 0; t < n_temps; ++t)
                metropolis_sweep(&cx, run, t, s, sr + (size_t)t * N, &Er[t],
                                 &macc[(size_t)run * n_temps + t]);
            int32_t m = INT32_MAX;
            for (int t = 0; t < n_temps; ++t) if (Er[t] < m) m = Er[t];
            if (m < best[run]) { best[run] = m; first[run] = (int32_t)s; }
            if (exchange_every > 0 && s % (uint32_t)exchange_every == 0)
                exchange_pass(&cx, run, s, sr, Er, xacc + (size_t)run * (n_temps > 1 ? n_temps - 1 : 0),
                              copy ? &w : NULL);
        }
    }
    ctx_close(&cx);
    return 0;
}

int or_pt_sweeps(int L, const int8_t *J, int n_temps, const double *betas, int n_runs,
                 uint32_t seed, uint32_t uid, int8_t *spins, int32_t *E, int32_t *best,
                 int32_t *first, uint64_t *macc, uint64_t *xacc, uint32_t sweep0,
                 int n_sweeps, int exchange_every)
{
    return or_pt_sweeps_walk(L, J, n_temps, betas, n_runs, seed, uid, spins, E, best, first, macc, xacc,
                             sweep0, n_sweeps, exchange_every, NULL, NULL, NULL, NULL);
}

/* One standalone exchange sweep of every run with counter sweep = `sweep`. */
int or_pt_exchange_walk(int L, const int8_t *J, int n_temps, const double *betas, int n_runs,
                        uint32_t seed, uint32_t uid, int8_t *spins, int32_t *E, uint64_t *xacc,
                        uint32_t sweep, int32_t *copy, uint64_t *hot, uint64_t *trips, uint8_t *state)
{
    pt_ctx cx;
    if (ctx_open(&cx, L, J, n_temps, betas, n_runs, seed, uid) != 0) { ctx_close(&cx); return -1; }
    for (int run = 0; run < n_runs; ++run) {
        walk_run w;
        if (copy) w = walk_of_run(n_temps, run, copy, hot, trips, state);
        exchange_pass(&cx, run, sweep, spins + (size_t)run * n_temps * cx.N,
                      E + (size_t)run * n_temps, xacc + (size_t)run * (n_temps > 1 ? n_temps - 1 : 0),
                      copy ? &w : NULL);
    }
    ctx_close(&cx);
    return 0;
}

int or_pt_exchange(int L, const int8_t *J, int n_temps, const double *betas, int n_runs,
                   uint32_t seed, uint32_t uid, int8_t *spins, int32_t *E, uint64_t *xacc,
                   uint32_t sweep)
{
    return or_pt_exchange_walk(L, J, n_temps, betas, n_runs, seed, uid, spins, E, xacc, sweep,
                               NULL, NULL, NULL, NULL);
}

/* ------------------------------------------------------------------ */
/* Time to solution.                                                    */
/* target == INT32_MAX means "the best energy any run found".           */
/* Run r hits if best[r] <= target and first[r] <= horizon; the TTS is  */
/* the ceil(R/2)-th smallest hit time (lower median), misses counting   */
/* as +inf; if that is +inf the instance is unsolved, TTS = horizon+1.  */
/* ------------------------------------------------------------------ */
void or_tts(int n_runs, const int32_t *best, const int32_t *first, int32_t target,
            int32_t horizon, int32_t *tts, int32_t *n_hit, int32_t *target_used)
{
    if (target == INT32_MAX) {
        target = INT32_MAX;
        for (int r = 0; r < n_runs; ++r) if (best[r] < target) target = best[r];
    }
    int64_t *v = malloc(sizeof(int64_t) * (size_t)(n_runs > 0 ? n_runs : 1));
    int hits = 0;
    const int64_t INF = INT64_MAX;
    for (int r = 0; r < n_runs; ++r) {
        int hit = best[r] <= target && first[r] <= horizon;
        v[r] = hit ? first[r] : INF;
        hits += hit;
    }
    /* insertion sort: plain and obviously correct */
    for (int a = 1; a < n_runs; ++a) {
        int64_t x = v[a]; int b = a - 1;
        while (b >= 0 && v[b] > x) { v[b + 1] = v[b]; --b; }
        v[b + 1] = x;
    }
    int m = (n_runs + 1) / 2;                 /* ceil(R/2), 1-based rank */
    int64_t med = n_runs > 0 ? v[m - 1] : INF;
    *tts = (med == INF) ? horizon + 1 : (int32_t)med;
    *n_hit = hits;
    *target_used = target;
    free(v);
}

/* A full TTS evaluation of one instance: fresh runs keyed by (seed, uid),
 * pass_mult*S sweeps, target = best energy of the pass, horizon S. */
int or_tts_eval(int L, const int8_t *J, int n_temps, const double *betas, int n_runs,
                uint32_t seed, uint32_t uid, int32_t S, int32_t pass_mult, int exchange_every,
                int32_t *tts, int32_t *n_hit, int32_t *target)
{
    int N = 8 * L * L;
    size_t nrep = (size_t)n_runs * n_temps;
    int8_t *spins = malloc(nrep * N);
    int32_t *E = malloc(sizeof(int32_t) * nrep);
    int32_t *best = malloc(sizeof(int32_t) * n_runs), *first = malloc(sizeof(int32_t) * n_runs);
    uint64_t *macc = calloc(nrep, sizeof(uint64_t));
    uint64_t *xacc = calloc((size_t)n_runs * (n_temps > 1 ? n_temps - 1 : 1), sizeof(uint64_t));
    or_pt_init_spins(L, n_temps, n_runs, seed, uid, spins);
    or_pt_start(L, J, n_temps, n_runs, spins, E, best, first);
    int rc = or_pt_sweeps(L, J, n_temps, betas, n_runs, seed, uid, spins, E, best, first,
                          macc, xacc, 0u, S * pass_mult, exchange_every);
    if (rc == 0) or_tts(n_runs, best, first, INT32_MAX, S, tts, n_hit, target);
    free(spins); free(E); free(best); free(first); free(macc); free(xacc);
    return rc;
}

/* A TTS evaluation under a doubling sweep budget (the reading used for the
 * large instances, where Sec. II's TTS needs a budget that grows with the
 * hardness, as the budget n of Appendix B does for HFS): fresh runs keyed by
 * (seed, uid) are run to S0 sweeps, then continued to 2 S0, 4 S0, ... up to
 * Smax.  At each level Lv the target is the best energy any run found within
 * Lv sweeps and the TTS is taken with horizon Lv; the first level with
 * TTS <= Lv / 4 gives the result (the target pass is then at least four
 * times the TTS, as with the fixed 4x pass).  If no level qualifies, the
 * instance is unsolved: TTS = Smax + 1, with the hits and target of the last
 * level.  *level receives the level that decided (Smax when unsolved).
 * Smax must be S0 times a power of two. */
int or_tts_eval_doubling(int L, const int8_t *J, int n_temps, const double *betas, int n_runs,
                         uint32_t seed, uint32_t uid, int32_t S0, int32_t Smax, int exchange_every,
                         int32_t *tts, int32_t *n_hit, int32_t *target, int32_t *level)
{
    int N = 8 * L * L;
    size_t nrep = (size_t)n_runs * n_temps;
    int8_t *spins = malloc(nrep * N);
    int32_t *E = malloc(sizeof(int32_t) * nrep);
    int32_t *best = malloc(sizeof(int32_t) * n_runs), *first = malloc(sizeof(int32_t) * n_runs);
    uint64_t *macc = calloc(nrep, sizeof(uint64_t));
    uint64_t *xacc = calloc((size_t)n_runs * (n_temps > 1 ? n_temps - 1 : 1), sizeof(uint64_t));
    or_pt_init_spins(L, n_temps, n_runs, seed, uid, spins);
    or_pt_start(L, J, n_temps, n_runs, spins, E, best, first);
    int rc = 0;
    int32_t done = 0;
    for (int32_t lv = S0;; lv *= 2) {
        rc = or_pt_sweeps(L, J, n_temps, betas, n_runs, seed, uid, spins, E, best, first,
                          macc, xacc, (uint32_t)done, lv - done, exchange_every);
        if (rc) break;
        done = lv;
        or_tts(n_runs, best, first, INT32_MAX, lv, tts, n_hit, target);
        *level = lv;
        if (*tts <= lv / 4) break;
        if (lv >= Smax) { *tts = Smax + 1; break; }
    }
    free(spins); free(E); free(best); free(first); free(macc); free(xacc);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Random adaptive optimisation (Algorithm 1).                          */
/* Proposal j of step t: one Philox call, key (seed, base_uid), counter */
/* (t, j, 0, 3): word 0 picks the coupler e = floor(w0 E / 2^32), word  */
/* 1 picks the new value among the five allowed values other than the   */
/* current one (floor(w1 5 / 2^32) into the ascending list), word 2 is  */
/* the candidate's PT key uid, word 3 the Boltzmann-acceptance uniform. */
/* ------------------------------------------------------------------ */
static const int8_t OR_JVALS[6] = {-3, -2, -1, 1, 2, 3};

void or_engineer_draw(int L, const int8_t *J, uint32_t seed, uint32_t base_uid, uint32_t step,
                      uint32_t proposal, int32_t *edge, int32_t *value, uint32_t *cand_uid,
                      uint32_t *u_accept)
{
    uint32_t ctr[4] = {step, proposal, 0u, 3u}, key[2] = {seed, base_uid}, w[4];
    or_philox4x32_10(ctr, key, w);
    uint32_t E = (uint32_t)or_chimera_n_edges(L);
    int e = (int)(((uint64_t)w[0] * E) >> 32);
    int pick = (int)(((uint64_t)w[1] * 5u) >> 32);
    int8_t allowed[5]; int na = 0;
    for (int a = 0; a < 6; ++a) if (OR_JVALS[a] != J[e] && na < 5) allowed[na++] = OR_JVALS[a];
    *edge = e;
    *value = allowed[pick];
    *cand_uid = w[2];
    *u_accept = w[3];
}

/* Acceptance of a candidate in Algorithm 1: a move that makes the instance
 * harder (direction +1) or easier (direction -1, the reversed optimisation
 * of Sec. III.A) is kept; otherwise it is kept with probability
 * exp(-beta_rao |TTS' - TTS|), decided by the uniform u < floor(p 2^32).
 * beta_rao < 0 stands for beta = infinity (greedy: never). */
int or_rao_accept(int32_t tts_cur, int32_t tts_new, int direction, double beta_rao, uint32_t u)
{
    int64_t gain = (int64_t)direction * ((int64_t)tts_new - (int64_t)tts_cur);
    if (gain > 0) return 1;
    if (beta_rao < 0.0) return 0;
    double dt = fabs((double)tts_new - (double)tts_cur);
    return u < prob_to_u32(exp(-beta_rao * dt));
}

/* Runs n_steps RAO steps t = step0 .. step0+n_steps-1 on J (in place).
 * tts_cur: in = TTS of the current J (if < 0 it is measured with uid = base_uid);
 * out = TTS of the final J.  beta_rao < 0 means greedy (beta = inf).
 * direction +1 maximises TTS (hard instances), -1 minimises it (Sec. III.A).
 * Per-step log arrays (length n_steps) may be NULL. */
/* One candidate's TTS: the fixed pass (pass_mult * S sweeps, horizon S) or,
 * with max_sweeps > 0, the doubling budget from S to max_sweeps. */
static int eval_budget(int L, const int8_t *J, int n_temps, const double *betas, int n_runs,
                       uint32_t seed, uint32_t uid, int32_t S, int32_t pass_mult, int32_t max_sweeps,
                       int exchange_every, int32_t *tts)
{
    int32_t nh, tg, lv;
    if (max_sweeps > 0)
        return or_tts_eval_doubling(L, J, n_temps, betas, n_runs, seed, uid, S, max_sweeps,
                                    exchange_every, tts, &nh, &tg, &lv);
    return or_tts_eval(L, J, n_temps, betas, n_runs, seed, uid, S, pass_mult, exchange_every,
                       tts, &nh, &tg);
}

int or_engineer_run_budget(int L, int8_t *J, int n_temps, const double *betas, int n_runs,
                           uint32_t seed, uint32_t base_uid, int32_t S, int32_t pass_mult,
                           int32_t max_sweeps, int exchange_every, uint32_t step0, int n_steps,
                           double beta_rao, int direction, int32_t *tts_cur,
                           int32_t *log_edge, int32_t *log_old, int32_t *log_new,
                           int32_t *log_tts, int32_t *log_accept)
{
    int32_t cur = *tts_cur;
    if (cur < 0) {
        int rc = eval_budget(L, J, n_temps, betas, n_runs, seed, base_uid, S, pass_mult, max_sweeps,
                             exchange_every, &cur);
        if (rc) return rc;
    }
    for (int a = 0; a < n_steps; ++a) {
        uint32_t t = step0 + (uint32_t)a;
        int32_t e, v; uint32_t cuid, uacc;
        or_engineer_draw(L, J, seed, base_uid, t, 0u, &e, &v, &cuid, &uacc);
        int8_t old = J[e];
        J[e] = (int8_t)v;
        int32_t tn;
        int rc = eval_budget(L, J, n_temps, betas, n_runs, seed, cuid, S, pass_mult, max_sweeps,
                             exchange_every, &tn);
        if (rc) { J[e] = old; return rc; }
        int accept = or_rao_accept(cur, tn, direction, beta_rao, uacc);
        if (accept) cur = tn; else J[e] = old;
        if (log_edge) log_edge[a] = e;
        if (log_old) log_old[a] = old;
        if (log_new) log_new[a] = v;
        if (log_tts) log_tts[a] = tn;
        if (log_accept) log_accept[a] = accept;
    }
    *tts_cur = cur;
    return 0;
}

int or_engineer_run(int L, int8_t *J, int n_temps, const double *betas, int n_runs,
                    uint32_t seed, uint32_t base_uid, int32_t S, int32_t pass_mult,
                    int exchange_every, uint32_t step0, int n_steps, double beta_rao,
                    int direction, int32_t *tts_cur,
                    int32_t *log_edge, int32_t *log_old, int32_t *log_new,
                    int32_t *log_tts, int32_t *log_accept)
{
    return or_engineer_run_budget(L, J, n_temps, betas, n_runs, seed, base_uid, S, pass_mult, 0,
                                  exchange_every, step0, n_steps, beta_rao, direction, tts_cur,
                                  log_edge, log_old, log_new, log_tts, log_accept);
}

/* Random adaptive optimisation with the adaptive budget of Appendix B.  The
 * paper's HFS evaluation repeats until the lowest energy has been found n+1
 * times; a step whose wall-clock time T_step exceeds T_max halves n (never
 * below 16, starting at 512), and beta = 6.5 n.  The deterministic
 * counterpart here: n is the number of PT runs an evaluation uses (runs
 * 0 .. n-1 of the instance's streams), the step's cost is n times the sweeps
 * the candidate's evaluation used (pass_mult * S, or the deciding level of
 * the doubling budget) in place of T_step, and after a step whose cost
 * exceeds cost_max the next step uses max(n_min, n / 2) runs.  The Boltzmann
 * branch uses beta = beta_per_run * n when beta_per_run > 0 (else the fixed
 * beta_rao).  *n_cur: in = runs of the next step, out = after the last step.
 * log_n / log_level (may be NULL): runs and sweeps of every step. */
int or_engineer_run_adaptive(int L, int8_t *J, int n_temps, const double *betas, uint32_t seed,
                             uint32_t base_uid, int32_t S, int32_t pass_mult, int32_t max_sweeps,
                             int exchange_every, uint32_t step0, int n_steps, double beta_rao,
                             double beta_per_run, int direction, int32_t n_min, int64_t cost_max,
                             int32_t *n_cur, int32_t *tts_cur, int32_t *log_edge, int32_t *log_new,
                             int32_t *log_tts, int32_t *log_accept, int32_t *log_n, int32_t *log_level)
{
    int32_t cur = *tts_cur, n = *n_cur;
    for (int a = 0; a < n_steps; ++a) {
        uint32_t t = step0 + (uint32_t)a;
        int32_t e, v; uint32_t cuid, uacc;
        or_engineer_draw(L, J, seed, base_uid, t, 0u, &e, &v, &cuid, &uacc);
        int8_t old = J[e];
        J[e] = (int8_t)v;
        int32_t tn, nh, tg, level;
        int rc;
        if (max_sweeps > 0) {
            rc = or_tts_eval_doubling(L, J, n_temps, betas, n, seed, cuid, S, max_sweeps, exchange_every,
                                      &tn, &nh, &tg, &level);
        } else {
            rc = or_tts_eval(L, J, n_temps, betas, n, seed, cuid, S, pass_mult, exchange_every, &tn, &nh, &tg);
            level = S * pass_mult;
        }
        if (rc) { J[e] = old; return rc; }
        double beta = beta_per_run > 0.0 ? beta_per_run * (double)n : beta_rao;
        int accept = or_rao_accept(cur, tn, direction, beta, uacc);
        if (accept) cur = tn; else J[e] = old;
        if (log_edge) log_edge[a] = e;
        if (log_new) log_new[a] = v;
        if (log_tts) log_tts[a] = tn;
        if (log_accept) log_accept[a] = accept;
        if (log_n) log_n[a] = n;
        if (log_level) log_level[a] = level;
        if ((int64_t)n * level > cost_max && n > n_min) n = n / 2 > n_min ? n / 2 : n_min;
    }
    *tts_cur = cur;
    *n_cur = n;
    return 0;
}

/* Exact ground-state energy by enumeration of the colour-0 spins: on the
 * bipartite Chimera graph the colour-1 spins are then independent, each
 * contributing -|h_i|.  Feasible while colour 0 has <= 24 spins (L <= 2). */
int32_t or_ground_energy_bipartite(int L, const int8_t *J)
{
    int N = 8 * L * L;
    nbr_list *nl = build_neighbours(L, J);
    int idx0[64], n0 = 0;
    for (int i = 0; i < N; ++i) if (or_spin_colour(L, i) == 0) idx0[n0++] = i;
    int8_t *s = calloc((size_t)N, 1);
    int32_t bestE = INT32_MAX;
    for (uint64_t m = 0; m < (1ull << n0); ++m) {
        for (int a = 0; a < n0; ++a) s[idx0[a]] = ((m >> a) & 1) ? -1 : 1;
        int32_t e = 0;
        for (int i = 0; i < N; ++i) {
            if (or_spin_colour(L, i) != 1) continue;
            int h = 0;
            for (int a = 0; a < nl[i].n; ++a) h += nl[i].Jn[a] * s[nl[i].nb[a]];
            e -= h < 0 ? -h : h;
        }
        if (e < bestE) bestE = e;
    }
    free(s); free(nl);
    return bestE;
}

/* ------------------------------------------------------------------ */
/* Planted-solution instances and loop adaptive optimisation            */
/* (Sec. IV, Algorithm 2).                                              */
/* The instance is a sum of frustrated loops along Chimera edges, each   */
/* built to have the planted configuration as a ground state, so the     */
/* planted configuration is a ground state of the sum and                */
/* E_GS = sum over loops of -w (len - 2).  Readings (the loop rules are  */
/* only outlined in the paper): a loop is a simple cycle of length 4     */
/* (probability 0.1) or 6, weight w uniform in 1..w_max; every edge is   */
/* satisfied by the planted state except one, frustrated, edge.          */
/* Couplers of overlapping loops add, without a cap of their own; a       */
/* placement is redrawn only if it would take a coupler outside          */
/* [-127, 127] or a spin's sum of |J| above 127 (the representable        */
/* range of the couplers and local fields), which the paper's parameters  */
/* (weights 1..5, 350 loops on 512 spins) do not reach.                  */
/* Draws use key (seed, uid), kind 4:                                    */
/*   planted spin i: counter (0, 0xFFFFFFF0, i>>2, 4), word i&3, s = -1  */
/*     if the top bit is set;                                            */
/*   loop (c0, c1), attempt a: words j = 0..15 from counters             */
/*     (c0, c1, a<<2 | j>>2, 4): j0 of attempt 0 fixes the length for    */
/*     every attempt (u < floor(0.1 2^32) -> 4, else 6, the size chosen  */
/*     before the placement), j1 start vertex floor(u N / 2^32), j2..    */
/*     the walk (neighbour                                               */
/*     floor(u deg / 2^32) in ascending vertex order), j8 weight          */
/*     1 + floor(u w_max / 2^32), j9 frustrated position                 */
/*     floor(u len / 2^32); an attempt that revisits a vertex, does not  */
/*     close, or overflows a coupler is rejected;                        */
/*   initial loop m: (c0, c1) = (0, m); step t: removed loop             */
/*     floor(w0 M / 2^32), Boltzmann uniform w1 and candidate PT key w2  */
/*     from counter (t, 0xFFFFFFFE, 0, 4), the new loop (c0, c1) =       */
/*     (t, 0xFFFFFFFF); the initial instance's PT key is w2 of step 0.   */
/* A loop record is {len, w, frustrated position, edges[6] (-1 unused)}. */
/* ------------------------------------------------------------------ */
#define OR_LOOP_WORDS 9
#define OR_LAO_P4 429496730u
#define OR_LAO_ATTEMPTS (1 << 16)

typedef struct { int N, E; int32_t *ei, *ej; int deg[2048]; int nb[2048][6]; int ne[2048][6]; } or_lgraph;

static or_lgraph *lgraph_open(int L)
{
    or_lgraph *g = calloc(1, sizeof(or_lgraph));
    g->N = 8 * L * L;
    g->E = or_chimera_n_edges(L);
    g->ei = malloc(sizeof(int32_t) * g->E);
    g->ej = malloc(sizeof(int32_t) * g->E);
    or_chimera_edges(L, g->ei, g->ej);
    for (int e = 0; e < g->E; ++e) {
        int a = g->ei[e], b = g->ej[e];
        g->nb[a][g->deg[a]] = b; g->ne[a][g->deg[a]++] = e;
        g->nb[b][g->deg[b]] = a; g->ne[b][g->deg[b]++] = e;
    }
    for (int v = 0; v < g->N; ++v)                    /* ascending neighbour order */
        for (int i = 1; i < g->deg[v]; ++i)
            for (int k = i; k > 0 && g->nb[v][k - 1] > g->nb[v][k]; --k) {
                int t = g->nb[v][k]; g->nb[v][k] = g->nb[v][k - 1]; g->nb[v][k - 1] = t;
                t = g->ne[v][k]; g->ne[v][k] = g->ne[v][k - 1]; g->ne[v][k - 1] = t;
            }
    return g;
}

static void lgraph_close(or_lgraph *g) { free(g->ei); free(g->ej); free(g); }

static int lgraph_edge(const or_lgraph *g, int a, int b)
{
    for (int k = 0; k < g->deg[a]; ++k) if (g->nb[a][k] == b) return g->ne[a][k];
    return -1;
}

static uint32_t mulhi32(uint32_t u, uint32_t n) { return (uint32_t)(((uint64_t)u * n) >> 32); }

/* Coupler contribution of a loop record to its m-th edge. */
static int loop_term(const or_lgraph *g, const int8_t *planted, const int32_t *rec, int m)
{
    int e = rec[3 + m];
    int sgn = (m == rec[2]) ? 1 : -1;
    return sgn * rec[1] * planted[g->ei[e]] * planted[g->ej[e]];
}

static void loop_apply(const or_lgraph *g, const int8_t *planted, const int32_t *rec, int8_t *J, int sign)
{
    for (int m = 0; m < rec[0]; ++m) J[rec[3 + m]] = (int8_t)(J[rec[3 + m]] + sign * loop_term(g, planted, rec, m));
}

static int lao_draw_loop(const or_lgraph *g, const int8_t *planted, const int8_t *J, uint32_t seed,
                         uint32_t uid, uint32_t c0, uint32_t c1, int w_max, int32_t *rec)
{
    const int len = draw(seed, uid, c0, c1, 0u, 4u, 0) < OR_LAO_P4 ? 4 : 6;   /* fixed for every attempt */
    for (uint32_t a = 0; a < OR_LAO_ATTEMPTS; ++a) {
        uint32_t u[16];
        for (int j = 0; j < 16; ++j) u[j] = draw(seed, uid, c0, c1, (a << 2) | (uint32_t)(j >> 2), 4u, j & 3);
        int v[6], ok = 1;
        v[0] = (int)mulhi32(u[1], (uint32_t)g->N);
        for (int m = 1; m < len && ok; ++m) {
            int p = v[m - 1];
            v[m] = g->nb[p][mulhi32(u[1 + m], (uint32_t)g->deg[p])];
            for (int q = 0; q < m; ++q) if (v[q] == v[m]) ok = 0;
        }
        if (!ok) continue;
        int32_t r[OR_LOOP_WORDS];
        r[0] = len;
        r[1] = 1 + (int)mulhi32(u[8], (uint32_t)w_max);
        r[2] = (int)mulhi32(u[9], (uint32_t)len);
        for (int m = 0; m < 6; ++m) r[3 + m] = -1;
        for (int m = 0; m < len; ++m) {
            r[3 + m] = lgraph_edge(g, v[m], v[(m + 1) % len]);
            if (r[3 + m] < 0) ok = 0;
        }
        if (!ok) continue;
        int Jt[6];
        for (int m = 0; m < len && ok; ++m) {
            Jt[m] = J[r[3 + m]] + loop_term(g, planted, r, m);
            if (Jt[m] < -127 || Jt[m] > 127) ok = 0;
        }
        for (int m = 0; m < len && ok; ++m) {          /* every loop vertex's sum of |J| */
            int x = v[m], sum = 0;
            for (int k = 0; k < g->deg[x]; ++k) {
                int e = g->ne[x][k], val = J[e];
                for (int q = 0; q < len; ++q) if (r[3 + q] == e) val = Jt[q];
                sum += val < 0 ? -val : val;
            }
            if (sum > OR_KMAX_LIMIT) ok = 0;
        }
        if (!ok) continue;
        memcpy(rec, r, sizeof(r));
        return 0;
    }
    return -1;
}

static int32_t loops_gs(const int32_t *loops, int n_loops)
{
    int32_t e = 0;
    for (int m = 0; m < n_loops; ++m) e -= loops[m * OR_LOOP_WORDS + 1] * (loops[m * OR_LOOP_WORDS] - 2);
    return e;
}

int or_lao_plant(int L, uint32_t seed, uint32_t uid, int n_loops, int w_max, int8_t *planted,
                 int32_t *loops, int8_t *J, int32_t *E_gs)
{
    or_lgraph *g = lgraph_open(L);
    for (int i = 0; i < g->N; ++i)
        planted[i] = (draw(seed, uid, 0u, 0xFFFFFFF0u, (uint32_t)(i >> 2), 4u, i & 3) >> 31) ? -1 : 1;
    memset(J, 0, (size_t)g->E);
    for (int m = 0; m < n_loops; ++m) {
        if (lao_draw_loop(g, planted, J, seed, uid, 0u, (uint32_t)m, w_max, loops + m * OR_LOOP_WORDS)) {
            lgraph_close(g);
            return -1;
        }
        loop_apply(g, planted, loops + m * OR_LOOP_WORDS, J, 1);
    }
    *E_gs = loops_gs(loops, n_loops);
    lgraph_close(g);
    return 0;
}

/* PT-TTS against a known target (pass of S sweeps, horizon S). */
static int tts_known(int L, const int8_t *J, int n_temps, const double *betas, int n_runs, uint32_t seed,
                     uint32_t uid, int32_t S, int exchange_every, int32_t target, int32_t *tts)
{
    int N = 8 * L * L;
    size_t nrep = (size_t)n_runs * n_temps;
    int8_t *spins = malloc(nrep * N);
    int32_t *E = malloc(sizeof(int32_t) * nrep);
    int32_t *best = malloc(sizeof(int32_t) * n_runs), *first = malloc(sizeof(int32_t) * n_runs);
    uint64_t *macc = calloc(nrep, sizeof(uint64_t));
    uint64_t *xacc = calloc((size_t)n_runs * (n_temps > 1 ? n_temps - 1 : 1), sizeof(uint64_t));
    or_pt_init_spins(L, n_temps, n_runs, seed, uid, spins);
    or_pt_start(L, J, n_temps, n_runs, spins, E, best, first);
    int rc = or_pt_sweeps(L, J, n_temps, betas, n_runs, seed, uid, spins, E, best, first, macc, xacc, 0u, S,
                          exchange_every);
    int32_t nh, tg;
    if (rc == 0) or_tts(n_runs, best, first, target, S, tts, &nh, &tg);
    free(spins); free(E); free(best); free(first); free(macc); free(xacc);
    return rc;
}

/* LAO steps step0 .. step0+n_steps-1 (step0 >= 1) in place on (loops, J,
 * E_gs, tts_cur); tts_cur < 0 on entry: evaluate the instance first (key w2
 * of step 0).  Acceptance as in Algorithm 1 (direction, beta_rao < 0:
 * greedy).  Per step the logs get the removed loop, the candidate's TTS,
 * ground-state energy and acceptance (any log may be NULL). */
int or_lao_run(int L, int n_temps, const double *betas, int n_runs, uint32_t seed, uint32_t uid, int n_loops,
               int w_max, int32_t S, int exchange_every, double beta_rao, int direction, uint32_t step0,
               int n_steps, const int8_t *planted, int32_t *loops, int8_t *J, int32_t *E_gs, int32_t *tts_cur,
               int32_t *log_removed, int32_t *log_tts, int32_t *log_egs, int32_t *log_accept)
{
    or_lgraph *g = lgraph_open(L);
    int rc = 0;
    int8_t *Jc = malloc((size_t)g->E);
    if (*tts_cur < 0) {
        uint32_t u0 = draw(seed, uid, 0u, 0xFFFFFFFEu, 0u, 4u, 2);
        rc = tts_known(L, J, n_temps, betas, n_runs, seed, u0, S, exchange_every, *E_gs, tts_cur);
    }
    for (int a = 0; a < n_steps && rc == 0; ++a) {
        uint32_t t = step0 + (uint32_t)a;
        uint32_t ctl[3];
        for (int w = 0; w < 3; ++w) ctl[w] = draw(seed, uid, t, 0xFFFFFFFEu, 0u, 4u, w);
        int r = (int)mulhi32(ctl[0], (uint32_t)n_loops);
        int32_t *old = loops + r * OR_LOOP_WORDS, rec[OR_LOOP_WORDS];
        memcpy(Jc, J, (size_t)g->E);
        loop_apply(g, planted, old, Jc, -1);
        if (lao_draw_loop(g, planted, Jc, seed, uid, t, 0xFFFFFFFFu, w_max, rec)) { rc = -1; break; }
        loop_apply(g, planted, rec, Jc, 1);
        int32_t eg = *E_gs + old[1] * (old[0] - 2) - rec[1] * (rec[0] - 2), tn;
        rc = tts_known(L, Jc, n_temps, betas, n_runs, seed, ctl[2], S, exchange_every, eg, &tn);
        if (rc) break;
        int accept = or_rao_accept(*tts_cur, tn, direction, beta_rao, ctl[1]);
        if (accept) {
            memcpy(J, Jc, (size_t)g->E);
            memcpy(old, rec, sizeof(rec));
            *E_gs = eg;
            *tts_cur = tn;
        }
        if (log_removed) log_removed[a] = r;
        if (log_tts) log_tts[a] = tn;
        if (log_egs) log_egs[a] = eg;
        if (log_accept) log_accept[a] = accept;
    }
    free(Jc);
    lgraph_close(g);
    return rc;
}
