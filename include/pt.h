/*
 * pt.h -- C ABI of the GB300 parallel-tempering hardness engine.
 *
 * Method: "Practical engineering of hard spin-glass instances" (Marshall,
 * Martin-Mayor, Hen; arXiv:1605.03607).  An instance is a coupler vector J on
 * the ideal Chimera graph C_L (Appendix A, Fig. 8: L x L unit cells of K_{4,4},
 * N = 8 L^2 spins).  Its cost is the Ising energy H = sum_<ij> J_ij s_i s_j,
 * minimised over s_i = +-1 (Eq. 1, no fields).  Its hardness is measured by
 * parallel tempering (Sec. II: N_T copies at fixed temperatures, Metropolis
 * updates, neighbour temperature swaps obeying detailed balance) as a time to
 * solution in sweeps (Sec. II "TTS"), and the random adaptive optimisation
 * loop (Algorithm 1) perturbs one coupler at a time and keeps a perturbation
 * when the instance got harder.
 *
 * Conventions (all functions):
 *   - Every function returns PT_OK (0) or a PT_ERR_* code; on error the handle
 *     is unchanged unless stated, and pt_last_error() describes the failure.
 *   - Handles are opaque.  The library owns all device memory it allocates.
 *     Caller arrays are host pointers, read or written during the call only;
 *     nothing is retained after a call returns.
 *   - `stream` is a cudaStream_t (NULL: the library creates its own
 *     non-blocking stream).  Calls that return results synchronise that stream
 *     only, never the whole device.
 *   - Spin index i = 8 (r L + c) + 4 u + k with cell row r, column c in [0, L),
 *     u = 0 (vertical) / 1 (horizontal), k in [0, 4).  Coupler order: the 16
 *     intra-cell couplers of each cell (cell-major, then k of the vertical
 *     spin, then k of the horizontal spin), then the vertical inter-cell
 *     couplers (r, c, 0, k)-(r+1, c, 0, k) ordered by (r, c, k), then the
 *     horizontal ones (r, c, 1, k)-(r, c+1, 1, k) ordered by (r, c, k):
 *     16 L^2 + 8 L (L - 1) couplers.  J values are int8 in [-127, 127], and
 *     every spin's sum of |J| over its couplers must be <= 127 (the largest
 *     local field, which sizes the Metropolis table).  Random instances use
 *     {+-1, +-2, +-3}; planted instances (Sec. IV) sum loop weights.
 *   - Temperature slots t = 0 .. N_T-1 hold inverse temperatures beta_t,
 *     strictly descending (slot 0 is the coldest).
 *   - Random numbers are Philox4x32-10 (Salmon et al., SC'11) with key
 *     (seed, uid) and counter (sweep, run << 16 | slot, group, kind): kind 0
 *     Metropolis (group = i >> 2, word i & 3), 1 exchange (group = p >> 2,
 *     word p & 3, slot field 0), 2 initial spins, 3 engineering draws.
 */
#ifndef GB300_PT_H
#define GB300_PT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PT_OK 0
#define PT_ERR_ARG 1      /* invalid argument (sizes, ranges, ladder order, NULL) */
#define PT_ERR_CUDA 2     /* a CUDA runtime call failed; the handle should be destroyed */
#define PT_ERR_TIMEOUT 3  /* a bounded device wait gave up */
#define PT_ERR_OOM 4      /* device or host allocation failed */
#define PT_ERR_STATE 5    /* call not valid in the handle's current state */

#define PT_TARGET_BEST INT32_MAX   /* pt_tts target: the best energy any run found */
#define PT_KMAX 18                 /* largest |local field| of couplers in {+-1, +-2, +-3} */
#define PT_KMAX_LIMIT 127          /* largest |local field| any instance may have */

typedef struct pt_handle pt_handle;

/* Message for the last failure on `h` (or of the last failed pt_create when
 * h is NULL).  Static storage owned by the library; never NULL. */
const char *pt_last_error(const pt_handle *h);

/* Creates one instance with n_runs independent PT runs of n_temps slots
 * (Sec. II).  J: n_edges int8 couplers in the order above (n_edges must equal
 * 16 L^2 + 8 L (L - 1)); betas: n_temps doubles, strictly descending, > 0.
 * Builds on the host, in FP64, the Metropolis table thr[t][k] =
 * floor(exp(-2 k beta_t) 2^32) (k = 1..18) and the exchange tables
 * xthr[p][h] = floor(exp(-2 h (beta_p - beta_{p+1})) 2^32) (h = 1..H_p, H_p
 * the last nonzero entry), then draws the initial spins of every (run, slot)
 * from the kind-2 stream of (seed, instance_uid).  Limits: 1 <= L <= 16,
 * 1 <= n_temps <= 64, 1 <= n_runs <= 1024.  Errors: PT_ERR_ARG, PT_ERR_OOM,
 * PT_ERR_CUDA (no handle is returned). */
int pt_create(pt_handle **h, int32_t chimera_L, const int8_t *J, int32_t n_edges,
              const double *betas, int32_t n_temps, int32_t n_runs, uint32_t seed,
              uint32_t instance_uid, void *stream);

/* An Ising graph given by its coupler list (Eq. 1).  The kernels work on the
 * Chimera graph C_L (Appendix A), so the list must be a set of couplers of
 * C_L: n = 8 L^2 spins, every (ei[e], ej[e]) a Chimera coupler (either
 * orientation), none repeated.  Couplers of C_L that are not listed are zero:
 * this is how a device with inoperative qubits, such as the paper's 504 of 512
 * (Fig. 8), is described.  ei == ej == NULL means the full C_L in the coupler
 * order above (then n_edges = 16 L^2 + 8 L (L - 1)). */
typedef struct pt_graph {
    int32_t n, n_edges;
    const int32_t *ei, *ej;   /* n_edges endpoints, read during pt_create_graph only */
    int32_t chimera_L;
} pt_graph;

/* pt_create for a graph given as a coupler list: J [n_edges] in the list's
 * order is placed on the listed couplers (pt_get_couplers then returns the
 * full C_L vector in the library's order).  Errors as pt_create, plus
 * PT_ERR_ARG for a coupler that is not an edge of C_L, a repeated one, or
 * n != 8 L^2. */
int pt_create_graph(pt_handle **h, const pt_graph *g, const int8_t *J, const double *betas, int32_t n_temps,
                    int32_t n_runs, uint32_t seed, uint32_t instance_uid, void *stream);

/* Frees every device and host resource of h (NULL is ignored). */
void pt_destroy(pt_handle *h);

/* Fresh runs: redraws the initial spins from (seed, instance_uid), identity
 * slot-to-configuration map, full energies, best = min over slots, first = 0,
 * zero acceptance counters, sweep counter 0. */
int pt_reset(pt_handle *h, uint32_t instance_uid);

/* Replaces every configuration (host int8 +-1 array [n_runs][n_temps][N] in
 * slot order), then proceeds as pt_reset without redrawing spins (the sweep
 * counter is kept).  Used for gauge checks and resumption.  PT_ERR_ARG if a
 * value is not +-1. */
int pt_set_spins(pt_handle *h, const int8_t *spins);

/* Performs sweeps s = sweep+1 .. sweep+n_sweeps.  Each sweep is a full-lattice
 * checkerboard Metropolis sweep of every copy (colour (r + c + u) mod 2 = 0
 * first; Sec. III.B "full-lattice Metropolis sweeps"), then the per-run best
 * energy / first sweep update, then, when exchange_every > 0 and
 * s % exchange_every == 0, one exchange sweep over pairs p = 0..N_T-2 in
 * ascending order with acceptance min(1, exp((beta_p - beta_{p+1})
 * (E_p - E_{p+1}))) (Sec. II, detailed balance).  0 <= n_sweeps <= 2^24. */
int pt_sweep(pt_handle *h, int32_t n_sweeps, int32_t exchange_every);

/* One standalone exchange sweep with counter sweep = the current sweep count
 * (identical to the exchange pt_sweep performs after that sweep). */
int pt_exchange(pt_handle *h);

/* Copies the state to host arrays (any may be NULL):
 *   spins [n_runs][n_temps][N] in slot order, E [n_runs][n_temps] slot order,
 *   perm  [n_runs][n_temps]    configuration buffer held by each slot,
 *   best, first [n_runs]       lowest energy seen and the sweep it was first seen,
 *   macc  [n_runs][n_temps]    accepted Metropolis flips per slot,
 *   xacc  [n_runs][n_temps-1]  accepted exchanges per pair,
 *   sweep                      sweeps performed since the last reset. */
int pt_get_state(pt_handle *h, int8_t *spins, int32_t *E, uint8_t *perm, int32_t *best,
                 int32_t *first, uint64_t *macc, uint64_t *xacc, uint64_t *sweep);

/* Time to solution from the current state (Sec. II "TTS"): target T =
 * E_target, or the lowest best energy over runs when E_target ==
 * PT_TARGET_BEST.  Run r hits when best[r] <= T and first[r] <= horizon; the
 * TTS is the ceil(R/2)-th smallest hit sweep (misses count as +inf) or
 * horizon + 1 ("unsolved") when fewer than ceil(R/2) runs hit.  The reduction
 * runs on the device.  Outputs are host pointers (n_hit, target_used may be
 * NULL). */
int pt_tts(pt_handle *h, int32_t E_target, int32_t horizon, int32_t *tts, int32_t *n_hit,
           int32_t *target_used);

/* A full PT-TTS evaluation: pt_reset(uid), pass_mult * S sweeps with exchange
 * every `exchange_every` sweeps, then pt_tts(PT_TARGET_BEST, horizon = S).
 * With pass_mult = 4 the target is the best energy of a 4x longer pass of the
 * same runs and only hits within the first S sweeps count. */
int pt_tts_eval(pt_handle *h, uint32_t uid, int32_t S, int32_t pass_mult,
                int32_t exchange_every, int32_t *tts, int32_t *n_hit, int32_t *target);

/* Sets coupler `edge` to `value` (|value| <= 127, every spin's sum of |J|
 * still <= 127), recomputes the energies of the current configurations and
 * restarts the best/first record from them (best = min over slots, first =
 * current sweep).  A change that needs a larger Metropolis table enlarges it
 * (pt_get_table_rows). */
int pt_set_coupler(pt_handle *h, int32_t edge, int8_t value);

/* Copies the current couplers (n_edges int8) to the host. */
int pt_get_couplers(pt_handle *h, int8_t *J);

/* Copies the host-built acceptance tables: thr [n_temps][rows] with rows
 * from pt_get_table_rows (entry k = 0 unused; row k = floor(exp(-2 k beta)
 * 2^32)), xoff [n_temps] (pair p owns xthr[xoff[p] .. xoff[p+1]-1] for
 * h = 1..H_p), xthr (capacity xthr_cap entries; may be NULL to query), and the
 * total exchange-table length in *xthr_len. */
int pt_get_tables(const pt_handle *h, uint32_t *thr, int64_t *xoff, uint32_t *xthr,
                  int64_t xthr_cap, int64_t *xthr_len);

/* Debug builds.  A library compiled with -DPT_DEBUG (build(debug=True):
 * libpt_gb300_debug.so) checks every data-dependent shared- and global-memory
 * index of its kernels: table rows, slot-map entries, exchange-table ranges,
 * run indexes, neighbour words.  A failed check records a code in a device
 * word and the access goes to index 0 instead, so no kernel faults or leaves
 * a barrier early; after every launch the host synchronises the stream, reads
 * and clears the word and prints the first code to stderr.  pt_debug_enabled
 * returns 1 in such a build, 0 otherwise; pt_debug_status returns (and
 * clears) the first code seen since the last call, 0 if none (always 0 in a
 * release build).  Codes: 1 Metropolis table row, 2 slot map, 3 exchange
 * table range, 4 run index, 5 neighbour word, 6 more than 1024 runs in a
 * TTS reduction, 7 slot map in the energy kernel, 8 a closed-form exchange
 * criterion that differs from the table search (debug builds evaluate both),
 * 9 a bundle whose lattice side differs from its kernel's compile-time side. */
int pt_debug_enabled(void);
int pt_debug_status(uint32_t *code);

/* Rows per temperature of the Metropolis table (k = 0 .. rows-1): 19 for
 * couplers in {+-1, +-2, +-3}; otherwise the largest sum of |J| over a
 * spin's couplers plus one, rounded up to a multiple of 4.  It grows when a
 * coupler change or candidate needs more and never shrinks. */
int pt_get_table_rows(const pt_handle *h, int32_t *rows);

/* The paper has no counterpart to this entry point: it is pt_tts_eval for
 * callers that cannot allocate device memory at call time, for instance code
 * running inside another framework whose allocator or memory pool already
 * owns the GPU's memory (a new cudaMalloc would fail or fragment it), or
 * latency-critical loops that cannot take the device-wide synchronisation
 * cudaMalloc/cudaFree may cause.  It creates no handle and allocates nothing:
 * its device scratch is one static 4 MiB array that every GPU loading this
 * library holds until the process exits, and its host staging is static.
 * Same arguments and results as pt_create + pt_tts_eval (J, betas: host
 * arrays as in pt_create; tts, n_hit, target: host outputs, n_hit and target
 * may be NULL); the call synchronises `stream` (NULL: the legacy default
 * stream).  Limits: n_runs * n_temps * 8 L^2 <= 2^21, n_runs * n_temps <=
 * 16384, n_runs <= 1024, exchange tables <= 2^17 entries; larger problems
 * return PT_ERR_ARG and pt_last_error(NULL) says which limit was exceeded.
 * All calls share the scratch (each call re-initialises it); calls that
 * overlap on the GPU race.  The first call on a device resolves the
 * scratch's device address; make that first call before any stream capture. */
int pt_tts_eval_noalloc(int32_t chimera_L, const int8_t *J, int32_t n_edges, const double *betas,
                        int32_t n_temps, int32_t n_runs, uint32_t seed, uint32_t uid, int32_t S,
                        int32_t pass_mult, int32_t exchange_every, void *stream, int32_t *tts,
                        int32_t *n_hit, int32_t *target);

/* PT-TTS evaluation under a doubling sweep budget.  The TTS of Sec. II
 * needs a sweep budget that grows with the instance's hardness (the paper
 * adapts the HFS repeat count n for the same reason, Appendix B); here fresh
 * runs keyed by (seed, uid) run S0 sweeps and are then continued, on the
 * same random streams, to 2 S0, 4 S0, ... Smax.  At each level Lv the target
 * is the best energy any run found within Lv sweeps and the TTS is the lower
 * median first-hit sweep with horizon Lv (pt_tts); the first level with
 * TTS <= Lv / 4 gives the result (the target pass is then at least four
 * times the TTS).  If none does, *tts = Smax + 1 (unsolved) and n_hit /
 * target are those of level Smax.  *level: the deciding level.  Smax must be
 * S0 * 2^k (k >= 0), Smax <= 2^30.  Resets the handle's runs.  Any output
 * but tts may be NULL. */
int pt_tts_eval_doubling(pt_handle *h, uint32_t uid, int32_t S0, int32_t Smax, int32_t exchange_every,
                         int32_t *tts, int32_t *n_hit, int32_t *target, int32_t *level);

/* PT-TTS evaluations of k instances of the handle's shape in one batched
 * launch sequence: J holds k coupler vectors [k][n_edges] (values in
 * [-127, 127], every spin's sum of |J| <= 127), instance j uses PT key uids[j].  max_sweeps == 0: the fixed pass
 * of pt_tts_eval (pass_mult * S sweeps, horizon S); > 0: the doubling budget
 * of pt_tts_eval_doubling from S to max_sweeps.  Outputs have k entries;
 * level[j] is the deciding level (pass_mult * S for the fixed pass).  Only
 * tts is required.  The handle's own runs and loop state are untouched.
 * 1 <= k <= 256. */
int pt_tts_eval_many(pt_handle *h, int32_t k, const int8_t *J, const uint32_t *uids, int32_t S,
                     int32_t pass_mult, int32_t max_sweeps, int32_t exchange_every, int32_t *tts,
                     int32_t *n_hit, int32_t *target, int32_t *level);

/* Random adaptive optimisation (Algorithm 1). */
typedef struct {
    int32_t S;               /* TTS horizon in sweeps */
    int32_t pass_mult;       /* target pass length = pass_mult * S */
    int32_t exchange_every;  /* sweeps between exchange sweeps */
    int32_t direction;       /* +1: maximise TTS (hard instances); -1: minimise (easy) */
    double beta_rao;         /* < 0: greedy (keep only strict improvements); else
                                also keep a worse move with prob. exp(-beta |dTTS|) */
    int32_t max_sweeps;      /* 0: fixed budget (pass_mult * S sweeps, horizon S).
                                > 0: doubling budget S, 2S, 4S, ... <= max_sweeps on the
                                same runs (pt_tts_eval_doubling); max_sweeps = S * 2^k,
                                pass_mult must be 1; unsolved = max_sweeps + 1 */
} pt_rule;

typedef struct {
    int32_t edge, old_value, new_value;
    int32_t tts_old, tts_new, accepted;
    uint32_t cand_uid;
    int32_t n_runs;          /* PT runs the candidate's evaluation used */
    int32_t level;           /* sweeps it used: pass_mult * S, or the deciding doubling level */
} pt_step_result;

/* Starts a loop on the handle's current couplers: measures their TTS with
 * uid = base_uid (pt_tts_eval) and stores rule, base_uid and that TTS. */
int engineer_begin(pt_handle *h, const pt_rule *rule, uint32_t base_uid, int32_t *tts0);

/* One RAO step t: draws a coupler e = floor(w0 E / 2^32) and a new value
 * (floor(w1 5 / 2^32)-th of the five allowed values other than J_e, ascending)
 * from Philox key (seed, base_uid), counter (t, 0, 0, 3); evaluates the
 * candidate with uid = w2; keeps it if direction * (TTS' - TTS) > 0, or else
 * if beta_rao >= 0 and w3 < floor(exp(-beta_rao |TTS' - TTS|) 2^32).
 * Requires engineer_begin. */
int engineer_step(pt_handle *h, uint32_t step, pt_step_result *out);

/* n_steps consecutive steps t = step0 .. step0+n_steps-1 with results
 * identical to n_steps engineer_step calls.  `speculation` (1..16)
 * candidates are drawn against the current couplers and evaluated in one
 * batched launch; every candidate after the first kept one is discarded and
 * redrawn.  A batch is always evaluated in full, also when fewer steps remain
 * in the call; the evaluated candidates of the steps past the call's end are
 * kept and used by the next engineer_run call if it starts at the next step
 * and the couplers, runs per evaluation, pt_rule and base uid are unchanged
 * (engineer_begin, engineer_set_adaptive, pt_set_coupler, lao_*, the guided
 * step and pt_restore drop them).  out: n_steps results (may be NULL). */
int engineer_run(pt_handle *h, uint32_t step0, int32_t n_steps, int32_t speculation,
                 pt_step_result *out);

/* The adaptive budget of Appendix B for engineer_run.  The paper repeats HFS
 * until the lowest energy is found n+1 times, halves n (start 512, floor 16)
 * after a step whose wall-clock time exceeds T_max, and uses beta = 6.5 n.
 * Here n is the number of PT runs a candidate's evaluation uses (runs
 * 0 .. n-1 of its streams, so a smaller n is a prefix of a larger one), a
 * step's cost is n times the sweeps that evaluation used (pass_mult * S, or
 * the deciding level of the doubling budget) in place of T_step, and after a
 * step whose cost exceeds cost_max the next step uses max(n_min, n / 2) runs.
 * beta_per_run > 0 sets the Boltzmann beta of each step to beta_per_run * n
 * (else pt_rule.beta_rao applies).  A speculative batch is cut after the
 * candidate that halves n, like after a kept one, so results equal those of
 * single steps.  The current instance keeps the TTS it was measured with.
 * n0 = 0 switches the rule off; otherwise 1 <= n_min <= n0 <= n_runs. */
int engineer_set_adaptive(pt_handle *h, int32_t n0, int32_t n_min, int64_t cost_max, double beta_per_run);

/* Runs the next engineering step will use (n_runs without the adaptive rule). */
int engineer_adaptive_runs(const pt_handle *h, int32_t *n);

/* Current loop state: TTS of the current couplers. */
int engineer_current_tts(const pt_handle *h, int32_t *tts);

/* Current loop state of an engineering (Algorithm 1) or LAO (Algorithm 2)
 * loop: the TTS of the current instance and how many of its runs reached
 * the target in the evaluation that measured it (fewer than half: the TTS
 * is the unsolved value, horizon + 1, and no candidate can be kept by the
 * greedy rule).  Either pointer may be NULL.  PT_ERR_STATE before
 * engineer_begin / lao_begin. */
int engineer_current_state(const pt_handle *h, int32_t *tts, int32_t *n_hit);

/* ---------------------------------------------------------------------
 * Planted-solution instances and loop adaptive optimisation (Sec. IV,
 * Algorithm 2).  An instance is a sum of frustrated loops along Chimera
 * edges, each with the planted configuration as a ground state, so the
 * planted configuration is a ground state of the sum and its energy
 * E_GS = sum over loops of -w (len - 2) is known: PT-TTS evaluations use it
 * as the target (one pass of S sweeps).  Loops: simple cycles of length 4
 * (probability 0.1) or 6, weight w uniform in 1..w_max (the paper uses
 * integer weights in [1, 5]), every edge satisfied by the planted state
 * except one; couplers of overlapping loops add.  A placement that would take
 * a coupler outside [-127, 127] or a spin's sum of |J| above 127 (the
 * engine's int8 couplers and table bound) is redrawn; at the paper's
 * parameters no placement reaches these bounds.  Random draws: Philox kind 4 with key (seed, uid); the counters
 * are documented with lao_plant below.
 * --------------------------------------------------------------------- */
#define PT_LOOP_WORDS 9   /* loop record: len, w, frustrated position, edges[6] (-1 unused) */

typedef struct {
    int32_t removed;              /* index of the loop taken out */
    int32_t loop[PT_LOOP_WORDS];  /* the loop put in */
    int32_t E_gs_new;             /* the candidate's ground-state energy */
    int32_t tts_old, tts_new, accepted;
    uint32_t cand_uid;            /* the candidate's PT key */
} pt_lao_result;

/* Host-only (no GPU work): the planted state s (N = 8 L^2 values +-1; spin
 * i from counter (0, 0xFFFFFFF0, i>>2, 4), word i&3, -1 if its top bit is
 * set), n_loops loop records ([n_loops][PT_LOOP_WORDS]) placed one by one
 * (loop m: counters (0, m, a<<2 | j>>2, 4) for attempt a, words j: j0 of
 * attempt 0 the length, j1 the start vertex, j2.. the walk in ascending
 * neighbour order, j8 the weight, j9 the frustrated position), the summed
 * couplers J (n_edges, the order of pt_create) and E_GS.  PT_ERR_ARG for
 * bad sizes, PT_ERR_STATE if no admissible loop is found in 2^16 attempts. */
int lao_plant(int32_t chimera_L, uint32_t seed, uint32_t uid, int32_t n_loops, int32_t w_max,
              int8_t *planted, int32_t *loops, int8_t *J, int32_t *E_gs);

/* Replaces the handle's couplers by the planted instance (seed = the
 * handle's seed) and evaluates its TTS against E_GS (rule: S, exchange_every,
 * direction, beta_rao; pass_mult is ignored) with PT key w2 of counter
 * (0, 0xFFFFFFFE, 0, 4).  The handle is then in LAO mode (engineer_begin
 * switches it back). */
int lao_begin(pt_handle *h, const pt_rule *rule, uint32_t uid, int32_t n_loops, int32_t w_max,
              int32_t *tts0);

/* LAO steps step0 .. step0+n_steps-1 (step0 >= 1): step t removes loop
 * floor(w0 M / 2^32), puts in loop (t, 0xFFFFFFFF) drawn against the
 * remaining couplers, evaluates the candidate against its own E_GS with PT
 * key w2, and keeps it under Algorithm 1's rule (Boltzmann uniform w1); w0..w2
 * come from counter (t, 0xFFFFFFFE, 0, 4).  Candidates are PT-evaluated
 * `speculation` (1..16) at a time; results equal the step-by-step loop.  As in
 * engineer_run, a batch is always evaluated in full and the evaluations of
 * steps past the call's end are used by the next lao_run call if it starts at
 * the next step with the couplers, loops, E_GS and pt_rule unchanged.
 * out: n_steps records (may be NULL). */
int lao_run(pt_handle *h, uint32_t step0, int32_t n_steps, int32_t speculation, pt_lao_result *out);

/* Ground-state / first-excited-state overlaps (Sec. III.B) of the runs'
 * current replicas.  The first excited level *E1 is the lowest replica
 * energy above E_gs (INT32_MAX if none).  Samples: per run, its coldest
 * replica at energy E_gs (a ground state) and its coldest replica at *E1 (an
 * excited state), where present.  The overlap of two configurations is
 * 1 - 2 h / N (h: the Hamming distance), taken in absolute value (zero
 * fields: a configuration and its global flip are the same state).
 * *q_gs_gs: lower median over the distinct pairs of ground samples,
 * *q_gs_es: over all (ground, excited) pairs; -1 where there is no pair.  The
 * paper reports q_gs_es / q_gs_gs.  Pairwise distances are computed on the
 * GPU. */
int pt_overlaps(pt_handle *h, int32_t E_gs, int32_t *n_gs, int32_t *n_es, int32_t *E1, double *q_gs_gs,
                double *q_gs_es);

/* Current planted state (N), loops ([n_loops][PT_LOOP_WORDS]), couplers,
 * E_GS and TTS (any pointer may be NULL).  PT_ERR_STATE outside LAO mode. */
int lao_state(const pt_handle *h, int8_t *planted, int32_t *loops, int8_t *J, int32_t *E_gs, int32_t *tts);

/* Checkpoint of the complete PT state and couplers.  With buf == NULL only
 * *len is set; otherwise *len must be at least that size. */
int pt_checkpoint(pt_handle *h, void *buf, size_t *len);

/* Restores a checkpoint made by a handle with the same L, n_temps, n_runs and
 * ladder.  PT_ERR_ARG on a size or shape mismatch. */
int pt_restore(pt_handle *h, const void *buf, size_t len);

/* Launch schedule (results are identical for every valid choice):
 * slot_parallel = temperature slots one CTA processes concurrently per run
 * (threads per run = slot_parallel * L^2, a multiple of 32, <= 1024),
 * runs_per_cta = runs sharing one CTA, sweeps_per_launch = sweeps per kernel
 * launch.  0 keeps the current value. */
int pt_set_schedule(pt_handle *h, int32_t slot_parallel, int32_t runs_per_cta,
                    int32_t sweeps_per_launch);
int pt_get_schedule(const pt_handle *h, int32_t *slot_parallel, int32_t *runs_per_cta,
                    int32_t *sweeps_per_launch);

/* Thread mapping of the sweep kernel.  team == 0: cell-major (a thread owns
 * one Chimera cell and every slot_parallel-th temperature slot).  team > 0
 * (a power of two <= 32): slot-major, slot_parallel teams of `team` lanes per
 * run (>= 32 threads per run, <= 768 threads per CTA); a team owns every
 * slot_parallel-th spin buffer, updates it at the temperature of the slot
 * holding it, and its lanes split the cells, so the two colours are separated
 * by a team sync instead of a CTA barrier.  0 keeps slot_parallel /
 * runs_per_cta.  Results never depend on it. */
int pt_set_mapping(pt_handle *h, int32_t team, int32_t slot_parallel, int32_t runs_per_cta);
int pt_get_mapping(const pt_handle *h, int32_t *team);

/* Temperature random walk of every system copy (Sec. III.B).  A copy is one
 * configuration buffer (the slot map of pt_get_state points slots at
 * buffers); after pt_create, pt_reset, pt_tts_eval or pt_set_spins copy c is
 * the configuration that started in slot c.  After every exchange pass each
 * copy in the hot half (the
 * n_temps/2 highest temperatures, slots n_temps - n_temps/2 .. n_temps-1)
 * gets one more pass there; this is the statistic of the paper's first
 * mixing criterion (the copy spending the least time in the hot half spends
 * at least 20 % of the run there, time counted in exchange passes, i.e. in
 * elementary Monte Carlo steps of `exchange_every` sweeps + one exchange).
 * A copy completes a round trip when it is back in the coldest slot after
 * reaching the hottest slot since its previous visit to the coldest one.
 * pt_set_walk_stats(h, 1) allocates and zeroes the counters of this handle's
 * runs (PT_ERR_ARG if the current schedule has no shared memory left for
 * them), 0 frees them.  Counters restart on pt_reset, pt_tts_eval,
 * pt_set_spins and pt_restore.  Results of the runs never depend on it.
 * pt_get_walk_stats: hot and trips are host arrays of n_runs x n_temps
 * (run-major, by copy; either may be NULL), n_passes the exchange passes
 * counted since the counters restarted.  PT_ERR_STATE when not tracked. */
int pt_set_walk_stats(pt_handle *h, int32_t on);
int pt_get_walk_stats(pt_handle *h, uint64_t *hot, uint64_t *trips, uint64_t *n_passes);

/* Autotuner: times every feasible (slot_parallel, runs_per_cta in {1,2,4})
 * of both mappings (slot-major teams of 2..32 lanes, 1/8 .. all slots per
 * team) for `trial_sweeps` sweeps of a batch of n_inst (1..16) copies of this
 * instance, the shape of engineer_run's speculative batches, and keeps the
 * fastest.  The main runs are untouched; results never depend on the choice. */
int pt_autotune(pt_handle *h, int32_t n_inst, int32_t trial_sweeps);

/* Makes `device` the current device of the calling host thread for the
 * library's CUDA runtime (handles created afterwards live there).  Errors:
 * PT_ERR_ARG (index out of range), PT_ERR_CUDA; failures are reported by
 * pt_last_error(NULL). */
int pt_select_device(int32_t device);

/* Number of kernels this handle has launched so far. */
uint64_t pt_launch_count(const pt_handle *h);

/* Enables (on != 0) or disables CUDA-event timing of every sweep-kernel
 * launch, and zeroes the cumulative totals of pt_sweep_timing_total. */
int pt_set_timing(pt_handle *h, int on);

/* Cumulative device time (ms) and count of the timed sweep-kernel launches
 * since the last pt_set_timing. */
int pt_sweep_timing_total(const pt_handle *h, double *ms, uint64_t *launches);

/* Accounting of full PT-TTS evaluations (pt_tts_eval, engineer_*): instances
 * evaluated, batched evaluation rounds, and their device time in ms (CUDA
 * events from the first kernel of a round to its TTS reduction).  reset != 0
 * zeroes the counters after reading them. */
int pt_eval_stats(pt_handle *h, uint64_t *evals, uint64_t *batches, double *device_ms, int reset);

/* Device time of the sweep-kernel launches of the last pt_sweep/pt_tts_eval
 * call, summed (ms, CUDA events on the handle's stream), and their count. */
int pt_last_sweep_timing(const pt_handle *h, double *ms, int32_t *launches);

/* Integer-issue microbenchmark: the measured counterpart of the sweep
 * kernel's roofline peak (the sweep is bound by 32-bit integer instruction
 * issue; the paper has no counterpart).  Runs `kind` on the current device,
 * 8 CTAs of 256 threads per SM, each thread `iters` loop iterations of
 * independent dependency chains:
 *   0 LOP3 (three-input xor), 1 IMAD (32-bit multiply-add), 2 LOP3 and IMAD
 *   interleaved one to one, 3 DP4A (int8 dot product), each 8 operations per
 *   iteration; 4 Philox4x32-10 rounds of two states sharing one key schedule
 *   (4 widening multiplies, 4 three-input xors, 2 key adds: 10 operations).
 * One untimed launch, then `reps` launches timed with CUDA events on `stream`
 * (a cudaStream_t; NULL is the default stream).  Writes *ops_per_s (thread
 * operations per second over the whole device) and, if not NULL,
 * *ms_per_launch.  Allocates and frees one small device buffer.
 * Errors: PT_ERR_ARG (kind outside [0, 4], iters outside [1, 2^22], reps
 * outside [1, 1000], NULL ops_per_s), PT_ERR_OOM, PT_ERR_CUDA; failures are
 * reported by pt_last_error(NULL). */
int pt_int_issue_rate(int32_t kind, int32_t iters, int32_t reps, double *ops_per_s,
                      double *ms_per_launch, void *stream);

/* ---------------------------------------------------------------------
 * Batched PT: many instances of uneven size and temperature count, each
 * with n_runs independent runs (Sec. II), in one graph replay.  Instances
 * are grouped by Chimera size; each size has its own thread mapping,
 * schedule, CTA size and persistent grid, and the sizes run as concurrent
 * graph branches (largest work first by stream priority).
 * Instance i keeps its own key (seed, uid_i): its trajectory is identical to
 * a pt_create handle with the same (J, betas, n_runs, seed, uid).
 * --------------------------------------------------------------------- */
typedef struct {
    int32_t chimera_L;       /* 1..16 */
    int32_t n_temps;         /* 1..64 */
    const int8_t *J;         /* 16 L^2 + 8 L (L-1) int8 couplers (|J| <= 127, every spin's sum of
                                |J| <= 127), read during the call */
    const double *betas;     /* n_temps, strictly descending, > 0 */
    uint32_t uid;            /* second key word of this instance's random streams */
} pt_instance_desc;

typedef struct pt_batch pt_batch;

/* Message for the last failure on b (NULL: last failed pt_batch_create). */
const char *pt_batch_last_error(const pt_batch *b);

/* Copies the instances, builds their FP64 tables, allocates device state and
 * starts fresh runs (as pt_reset).  Errors: PT_ERR_ARG, PT_ERR_OOM, PT_ERR_CUDA. */
int pt_batch_create(pt_batch **b, int32_t n_inst, const pt_instance_desc *d, int32_t n_runs,
                    uint32_t seed, void *stream);
void pt_batch_destroy(pt_batch *b);

/* Fresh runs of every instance (spins from the kind-2 streams, sweep 0). */
int pt_batch_reset(pt_batch *b);

/* n_sweeps sweeps of every run of every instance (same sweep/exchange rule
 * as pt_sweep) as one replay of a CUDA graph holding the work-counter reset
 * and one persistent launch per size: a size's CTAs pull bundles of its runs,
 * longest first, from that size's atomic counter until none is left. */
int pt_batch_run(pt_batch *b, int32_t n_sweeps, int32_t exchange_every);

/* Per-instance TTS (rule of pt_tts with target = best found, horizon given):
 * tts, n_hit, target: host arrays of n_inst (n_hit, target may be NULL). */
int pt_batch_tts(pt_batch *b, int32_t horizon, int32_t *tts, int32_t *n_hit, int32_t *target);

/* State of instance `inst` in the layout of pt_get_state (any pointer may be NULL). */
int pt_batch_get_state(pt_batch *b, int32_t inst, int8_t *spins, int32_t *E, int32_t *best,
                       int32_t *first, uint64_t *macc, uint64_t *xacc);

/* Schedule of the instances of size chimera_L: slot_parallel slots
 * (cell-major: slot_parallel * L^2 threads per run) or teams (slot-major:
 * slot_parallel * team threads per run, at the size's largest temperature
 * count; an instance with fewer temperatures gets proportionally fewer
 * teams) per run, >= 32 threads per run, runs_per_cta runs per CTA, and the
 * CTA size `block` (a multiple of 32, <= 1024, <= 768 slot-major; 0: the
 * bundle's thread count rounded up to a warp).  chimera_L 0 sets `block` for
 * every size.  PT_ERR_ARG (nothing changed) when a size does not fit its
 * block or 227 KB of shared memory.  Results never depend on the schedule. */
int pt_batch_set_schedule(pt_batch *b, int32_t block, int32_t chimera_L, int32_t slot_parallel,
                          int32_t runs_per_cta);
int pt_batch_get_schedule(const pt_batch *b, int32_t chimera_L, int32_t *block,
                          int32_t *slot_parallel, int32_t *runs_per_cta);

/* Thread mapping of size chimera_L (the rule of pt_set_mapping): team 0 is
 * cell-major, team > 0 (a power of two <= 32) slot-major with slot_parallel
 * teams of `team` lanes per run.  Switching mapping starts from that mapping's
 * default schedule; slot_parallel / runs_per_cta 0 keep it; the CTA size
 * becomes the bundle's thread count.  chimera_L 0 gives every size the
 * mapping's default schedule.  PT_ERR_ARG (nothing changed) when the result
 * does not fit (>= 32 threads per run, <= 768 threads per CTA slot-major,
 * 227 KB of shared memory). */
int pt_batch_set_mapping(pt_batch *b, int32_t chimera_L, int32_t team, int32_t slot_parallel,
                         int32_t runs_per_cta);
int pt_batch_get_mapping(const pt_batch *b, int32_t chimera_L, int32_t *team);

/* Autotuner: size by size, times every feasible cell-major (slot_parallel,
 * runs_per_cta) and slot-major (team, slot_parallel, runs_per_cta) on all
 * instances of that size over `trial_sweeps` sweeps, with the CTA size the
 * bundle needs, keeps the fastest, then resets the runs.  *block (may be
 * NULL): the CTA size of the size with the most work. */
int pt_batch_autotune(pt_batch *b, int32_t trial_sweeps, int32_t *block);

/* Device time of the last pt_batch_run (CUDA events), persistent CTAs over
 * all sizes, largest CTA size, bundle count, kernels launched so far. */
int pt_batch_info(const pt_batch *b, double *last_run_ms, int32_t *grid, int32_t *block,
                  int32_t *n_bundles, uint64_t *launches);

/* ---------------------------------------------------------------------
 * Surrogate hardness model.  The paper has no surrogate: it is this
 * library's way to rank RAO proposals (Algorithm 1) so that only the most
 * promising ones get a PT-TTS evaluation (Sec. II TTS); PT stays the judge
 * of every kept move.  Message-passing network over the Chimera coupler
 * graph predicting log10 TTS:
 *   h0_i = X[u_i] (orientation), e0_e = Jt[idx(J_e)], idx: -3..-1,1..3 -> 0..5
 *   per layer: m_i = sum_{j in N(i)} relu(Wm [h_j, e_ij] + bm)
 *              h_i += relu(Wu [h_i, m_i] + bu); e_ij += relu(We [e_ij, h_i + h_j] + be)
 *   y = w2 . relu(W1 mean_i h_i + b1) + b2
 * Hidden width 64.  Parameters are one FP32 vector in the order X[2,64],
 * Jt[6,64], per layer Wm[64,128], bm, Wu[64,128], bu, We[64,128], be, then
 * W1[64,64], b1, w2, b2 (matrices row-major, rows = outputs).  Forward and
 * backward use BF16 weights/activations with FP32 accumulation (tensor
 * cores); master weights, gradients and Adam moments are FP32.
 * --------------------------------------------------------------------- */
typedef struct sg_model sg_model;

const char *sg_last_error(const sg_model *m);

/* hidden must be 64, 1 <= layers <= 8.  Parameters start at zero. */
int sg_create(sg_model **m, int32_t hidden, int32_t layers, void *stream);
void sg_destroy(sg_model *m);
int64_t sg_num_params(const sg_model *m);

/* Copies FP32 parameters in (resetting Adam) / out (host arrays of sg_num_params). */
int sg_set_params(sg_model *m, const float *theta);
int sg_get_params(sg_model *m, float *theta);

/* Predictions for B instances of C_L: J host [B][16 L^2 + 8 L (L-1)] with
 * values in {+-1, +-2, +-3}; y host [B]. */
int sg_forward(sg_model *m, int32_t L, int32_t B, const int8_t *J, float *y);

/* Mean squared error against targets t [B] and its gradient (host array of
 * sg_num_params, may be NULL). */
int sg_grad(sg_model *m, int32_t L, int32_t B, const int8_t *J, const float *t, float *loss, float *grad);

/* One Adam update (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) with
 * the gradient of the last sg_grad. */
int sg_adam(sg_model *m, float lr);

/* sg_grad followed by sg_adam. */
int sg_train_step(sg_model *m, int32_t L, int32_t B, const int8_t *J, const float *t, float lr, float *loss);

/* Kernels launched by this model so far. */
uint64_t sg_launch_count(const sg_model *m);

/* Surrogate-guided RAO step t (Algorithm 1 with a learned proposal filter):
 * draws n_prop proposals j = 0..n_prop-1 against the current couplers (the
 * draw of engineer_step with counter (t, j, 0, 3)), predicts their log10 TTS
 * with the surrogate m, PT-evaluates the `top` best-ranked ones (ties: lower
 * j first) in one batched launch, and keeps the one with the largest TTS
 * (ties: better rank) under the rule of engineer_step.  PT alone decides.
 * out: `top` results in rank order (accepted = 1 on the kept one, if any);
 * pred (may be NULL): the n_prop predictions; ranked (may be NULL): the
 * proposal indices of out.  1 <= top <= min(n_prop, 16), n_prop <= 1024.
 * Requires engineer_begin and couplers in {+-1, +-2, +-3}.
 * m == NULL: no ranking; proposals 0..top-1 are evaluated and kept under the
 * same best-of-top rule (the plain loop at identical acceptance, pred = 0). */
int engineer_guided_step(pt_handle *h, sg_model *m, uint32_t step, int32_t n_prop, int32_t top,
                         pt_step_result *out, float *pred, int32_t *ranked);

#ifdef __cplusplus
}
#endif
#endif
