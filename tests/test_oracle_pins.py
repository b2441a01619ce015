"""Pins of the CPU oracle against facts fixed outside it (no GPU needed).

Each test checks the oracle against something other than itself: published
known-answer vectors, closed forms, exhaustive enumeration, exact Boltzmann
statistics, or an exact symmetry of Eq. 1.
"""
import itertools
import math
import os
from decimal import Decimal, getcontext

import numpy as np
import pytest

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Philox4x32-10: published known-answer vectors (Salmon et al., SC'11).
# --------------------------------------------------------------------------
def test_philox_known_answers():
    n = 0
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        out = oracle.philox4x32_10(w[0:4], w[4:6])
        assert list(out) == w[6:10]
        n += 1
    assert n == 3


# --------------------------------------------------------------------------
# Chimera graph (Appendix A, Fig. 8): independent predicate-based adjacency.
# --------------------------------------------------------------------------
def _coords(L, i):
    cell, rem = divmod(i, 8)
    r, c = divmod(cell, L)
    u, k = divmod(rem, 4)
    return r, c, u, k


def _adjacent(L, i, j):
    r1, c1, u1, k1 = _coords(L, i)
    r2, c2, u2, k2 = _coords(L, j)
    if (r1, c1) == (r2, c2):
        return u1 != u2                                    # K_{4,4} inside a cell
    if u1 == u2 == 0 and c1 == c2 and abs(r1 - r2) == 1 and k1 == k2:
        return True                                        # vertical qubits couple along columns
    if u1 == u2 == 1 and r1 == r2 and abs(c1 - c2) == 1 and k1 == k2:
        return True                                        # horizontal qubits couple along rows
    return False


@pytest.mark.parametrize("L", [1, 2, 3, 4, 8])
def test_chimera_edges_match_predicate(L):
    ei, ej = oracle.chimera_edges(L)
    assert len(ei) == W.chimera_n_edges(L) == 16 * L * L + 8 * L * (L - 1)
    got = {(min(a, b), max(a, b)) for a, b in zip(ei, ej)}
    assert len(got) == len(ei)                             # no duplicates
    N = 8 * L * L
    if L <= 4:
        want = {(i, j) for i in range(N) for j in range(i + 1, N) if _adjacent(L, i, j)}
        assert got == want
    deg = np.bincount(np.concatenate([ei, ej]), minlength=N)
    assert deg.max() == {1: 4, 2: 5}.get(L, 6)          # every spin of C_2 sits on the boundary
    if L >= 3:                                             # interior cells: every spin has degree 6
        for i in range(N):
            r, c, u, k = _coords(L, i)
            if 0 < r < L - 1 and 0 < c < L - 1:
                assert deg[i] == 6


@pytest.mark.parametrize("L", [1, 4, 8])
def test_colouring_is_bipartition(L):
    ei, ej = oracle.chimera_edges(L)
    col = oracle.spin_colours(L)
    assert np.all(col[ei] != col[ej])
    for i in range(8 * L * L):                             # vertical (r+c)%2, horizontal (r+c+1)%2
        r, c, u, k = _coords(L, i)
        assert col[i] == ((r + c) % 2 if u == 0 else (r + c + 1) % 2)


# --------------------------------------------------------------------------
# Eq. 1 energy: dense matrix form, enumeration, symmetries.
# --------------------------------------------------------------------------
def _dense_J(L, J):
    N = 8 * L * L
    ei, ej = oracle.chimera_edges(L)
    A = np.zeros((N, N), np.int64)
    A[ei, ej] = J
    A[ej, ei] = J
    return A


def test_energy_matches_quadratic_form():
    rng = np.random.default_rng(3)
    for L in (1, 2, 4):
        J = W.random_couplers(L, 11, L)
        A = _dense_J(L, J)
        for _ in range(20):
            s = np.where(rng.integers(0, 2, 8 * L * L) == 0, -1, 1).astype(np.int8)
            assert oracle.energy(L, J, s) == int(s.astype(np.int64) @ A @ s) // 2
            assert oracle.energy(L, J, s) == oracle.energy(L, J, -s)   # global flip


def test_ground_state_enumeration_single_cell():
    for uid in range(5):
        J = W.random_couplers(1, 5, uid)
        states = np.array(list(itertools.product([-1, 1], repeat=8)), np.int8)
        E = [oracle.energy(1, J, s) for s in states]
        assert min(E) == oracle.ground_energy_bipartite(1, J)


def test_gauge_maps_energy():
    L = 4
    rng = np.random.default_rng(7)
    J = W.random_couplers(L, 2, 0)
    ei, ej = oracle.chimera_edges(L)
    g = np.where(rng.integers(0, 2, 8 * L * L) == 0, -1, 1).astype(np.int8)
    Jg = (g[ei] * g[ej] * J).astype(np.int8)
    for _ in range(10):
        s = np.where(rng.integers(0, 2, 8 * L * L) == 0, -1, 1).astype(np.int8)
        assert oracle.energy(L, Jg, g * s) == oracle.energy(L, J, s)


# --------------------------------------------------------------------------
# Acceptance tables: exact values at high precision.
# --------------------------------------------------------------------------
def _exact_u32(x_exponent: Decimal) -> tuple[int, Decimal]:
    v = (x_exponent.exp()) * (Decimal(2) ** 32)
    return int(v), v - int(v)


def test_metropolis_thresholds_exact():
    getcontext().prec = 60
    betas = W.beta_ladder(48, 0.05, 5.0)
    thr = oracle.metropolis_thresholds(betas)
    assert thr.shape == (48, 19)
    for t, b in enumerate(betas):
        for k in range(1, 19):
            want, frac = _exact_u32(-2 * k * Decimal(float(b)))
            if Decimal("1e-6") < frac < 1 - Decimal("1e-6"):
                assert int(thr[t, k]) == want, (t, k)
        assert np.all(np.diff(thr[t, 1:].astype(np.int64)) <= 0)


def test_exchange_thresholds_exact():
    getcontext().prec = 60
    betas = W.beta_ladder(16, 0.1, 3.0)
    off, table = oracle.exchange_thresholds(betas)
    for p in range(15):
        db = float(betas[p]) - float(betas[p + 1])
        seg = table[off[p]:off[p + 1]]
        H = len(seg)
        # H_p is the last h whose floor(exp(-2 h db) 2^32) is nonzero
        assert 2 * H * db <= 32 * math.log(2) + 1e-9 < 2 * (H + 1) * db + 1e-9
        assert np.all(seg > 0) and np.all(np.diff(seg.astype(np.int64)) <= 0)
        for h in (1, 2, H // 2 + 1, H):
            want, frac = _exact_u32(-2 * h * Decimal(db))
            if Decimal("1e-6") < frac < 1 - Decimal("1e-6"):
                assert int(seg[h - 1]) == want
    with pytest.raises(ValueError):
        oracle.exchange_thresholds(np.array([1.0, 1.0]))


# --------------------------------------------------------------------------
# Monte Carlo: incremental energy, exact Boltzmann statistics, gauge, GS.
# --------------------------------------------------------------------------
def test_incremental_energy_equals_recompute():
    L = 4
    J = W.random_couplers(L, 9, 1)
    st = oracle.PTState(L, J, W.beta_ladder(8, 0.1, 3.0), 3, seed=9, uid=1)
    assert np.array_equal(st.E, st.full_energies())
    for _ in range(5):
        st.sweeps(37, exchange_every=1)
        assert np.array_equal(st.E, st.full_energies())
    assert st.macc.sum() > 0 and st.xacc.sum() > 0
    assert np.all(st.best <= st.E.min(axis=1))


def _boltzmann(L, J, beta):
    states = np.array(list(itertools.product([-1, 1], repeat=8 * L * L)), np.int8)
    E = np.array([oracle.energy(L, J, s) for s in states], np.float64)
    w = np.exp(-beta * (E - E.min()))
    return states, E, w / w.sum()


def _state_index(spins):
    bits = (spins < 0).astype(np.int64)          # state order of itertools.product([-1, 1])
    return bits @ (1 << np.arange(bits.shape[-1] - 1, -1, -1))


def test_single_temperature_boltzmann_histogram():
    """A single K_{4,4} cell at one beta: the chain samples exp(-beta E)/Z."""
    L, beta, R = 1, 0.35, 64
    J = W.random_couplers(L, 21, 0)
    _, _, p = _boltzmann(L, J, beta)
    st = oracle.PTState(L, J, np.array([beta]), R, seed=21, uid=3)
    counts = np.zeros(256)
    for _ in range(3000):
        st.sweeps(1, exchange_every=0)
        np.add.at(counts, _state_index(st.spins[:, 0, :]), 1)
    n = counts.sum()
    chi2 = np.sum((counts - n * p) ** 2 / (n * p))
    assert chi2 / 255 < 3.0, chi2 / 255
    # a halved acceptance exponent (a plausible slip) is rejected by the same test
    _, _, p_wrong = _boltzmann(L, J, beta / 2)
    chi2_wrong = np.sum((counts - n * p_wrong) ** 2 / (n * p_wrong))
    assert chi2_wrong / 255 > 10 * max(chi2 / 255, 1.0)


def test_two_temperature_exchange_boltzmann():
    """PT with two slots: each slot must sample the Boltzmann law of its own beta
    (Sec. II: swaps obey detailed balance).  beta_0 is cold enough that it mixes
    only through exchanges with the hot slot."""
    L, R = 1, 64
    betas = np.array([1.1, 0.25])
    J = W.random_couplers(L, 31, 0)
    _, Es, p0 = _boltzmann(L, J, betas[0])
    _, _, p1 = _boltzmann(L, J, betas[1])
    st = oracle.PTState(L, J, betas, R, seed=31, uid=5)
    c0 = np.zeros(256)
    c1 = np.zeros(256)
    for _ in range(3000):
        st.sweeps(1, exchange_every=1)
        np.add.at(c0, _state_index(st.spins[:, 0, :]), 1)
        np.add.at(c1, _state_index(st.spins[:, 1, :]), 1)
    assert np.array_equal(st.E, st.full_energies())
    for c, p in ((c0, p0), (c1, p1)):
        n = c.sum()
        # compare energy-level distributions (robust at the cold slot)
        levels = np.unique(Es)
        obs = np.array([c[Es == e].sum() for e in levels]) / n
        exp_ = np.array([p[Es == e].sum() for e in levels])
        keep = exp_ > 1e-3
        assert np.max(np.abs(obs[keep] - exp_[keep])) < 0.02
    assert st.xacc.sum() > 0


def test_gauge_invariance_maps_trajectory():
    """J_ij -> g_i g_j J_ij with s -> g s maps every dE, acceptance and energy exactly."""
    L, R = 4, 3
    betas = W.beta_ladder(6, 0.2, 2.5)
    J = W.random_couplers(L, 41, 0)
    ei, ej = oracle.chimera_edges(L)
    colours = oracle.spin_colours(L)
    for g in (np.where(np.random.default_rng(1).integers(0, 2, 8 * L * L) == 0, -1, 1),
              np.where(colours == 0, 1, -1),              # bipartition gauge: J -> -J
              -np.ones(8 * L * L, np.int64)):             # global flip
        g = g.astype(np.int8)
        Jg = (g[ei] * g[ej] * J).astype(np.int8)
        a = oracle.PTState(L, J, betas, R, seed=41, uid=2)
        b = oracle.PTState(L, Jg, betas, R, seed=41, uid=2, spins=a.spins * g)
        for _ in range(3):
            a.sweeps(50, exchange_every=1)
            b.sweeps(50, exchange_every=1)
            assert np.array_equal(b.spins, a.spins * g)
            assert np.array_equal(a.E, b.E)
            assert np.array_equal(a.best, b.best) and np.array_equal(a.first, b.first)
            assert np.array_equal(a.macc, b.macc) and np.array_equal(a.xacc, b.xacc)
        if np.all(g == np.where(colours == 0, 1, -1)):
            assert np.array_equal(Jg, -J)


def test_pt_finds_exact_ground_state_two_by_two():
    L = 2
    for uid in range(3):
        J = W.random_couplers(L, 51, uid)
        gs = oracle.ground_energy_bipartite(L, J)
        st = oracle.PTState(L, J, W.beta_ladder(8, 0.1, 3.0), 8, seed=51, uid=uid)
        st.sweeps(2000, exchange_every=1)
        assert np.all(st.best == gs)
        assert np.all(st.best >= gs) and np.all(st.E >= gs)


def test_exchange_standalone_matches_fused():
    L = 4
    J = W.random_couplers(L, 61, 0)
    betas = W.beta_ladder(10, 0.1, 3.0)
    a = oracle.PTState(L, J, betas, 2, seed=61, uid=0)
    b = oracle.PTState(L, J, betas, 2, seed=61, uid=0)
    for _ in range(20):
        a.sweeps(1, exchange_every=1)
        b.sweeps(1, exchange_every=0)
        b.exchange()
    assert np.array_equal(a.spins, b.spins) and np.array_equal(a.xacc, b.xacc)


# --------------------------------------------------------------------------
# TTS: hand-constructed arrays.
# --------------------------------------------------------------------------
def test_tts_lower_median_closed_form():
    best = np.array([-10, -10, -10, -8, -10, -9, -10, -10], np.int32)
    first = np.array([50, 7, 900, 3, 20, 4, 100, 60], np.int32)
    # target = -10: hits at 50, 7, 900, 20, 100, 60 -> sorted 7,20,50,60,100,900,inf,inf; 4th = 60
    assert oracle.tts(best, first, oracle.TARGET_BEST, 1000) == (60, 6, -10)
    # horizon 55 drops 900,100,60 -> 7,20,50,inf.. ; 4th is inf -> unsolved = 56
    assert oracle.tts(best, first, oracle.TARGET_BEST, 55) == (56, 3, -10)
    # explicit looser target -9 also counts the run that found -9
    assert oracle.tts(best, first, -9, 1000) == (50, 7, -9)
    # odd R: ceil(3/2) = 2nd smallest
    assert oracle.tts(np.array([-2, -2, -2], np.int32), np.array([5, 1, 9], np.int32)) [0] == 5
    # R = 1
    assert oracle.tts(np.array([-4], np.int32), np.array([0], np.int32), oracle.TARGET_BEST, 10) == (0, 1, -4)


def test_tts_eval_is_prefix_of_longer_pass():
    """The 4x-pass reading: first[] of a run is a prefix property of its trajectory."""
    L = 4
    J = W.random_couplers(L, 71, 0)
    betas = W.beta_ladder(8, 0.1, 3.0)
    t4 = oracle.tts_eval(L, J, betas, 6, 71, 9, 256, 4, 1)
    st = oracle.PTState(L, J, betas, 6, seed=71, uid=9)
    st.sweeps(1024, 1)
    assert t4 == oracle.tts(st.best, st.first, oracle.TARGET_BEST, 256)


# --------------------------------------------------------------------------
# RAO (Algorithm 1).
# --------------------------------------------------------------------------
def test_engineer_draw_rules():
    L = 4
    J = W.random_couplers(L, 81, 0)
    seen_edges = set()
    for t in range(400):
        e, v, cu, ua = oracle.engineer_draw(L, J, 81, 0, t)
        assert 0 <= e < len(J) and v != J[e] and v in (-3, -2, -1, 1, 2, 3)
        seen_edges.add(e)
    assert len(seen_edges) > 200
    assert oracle.engineer_draw(L, J, 81, 0, 5) == oracle.engineer_draw(L, J, 81, 0, 5)


def test_engineer_run_replay_and_monotone():
    L = 4
    cfg = W.CONFIGS["c4_tiny"]
    J0 = W.random_couplers(L, cfg["seed"], 0)
    betas = W.beta_ladder(8, 0.1, 3.0)
    args = (L, J0, betas, 4, cfg["seed"], 0, 256, 1, 1, 1, 12)
    Ja, ta, la = oracle.engineer_run(*args)
    Jb, tb, lb = oracle.engineer_run(*args)
    assert ta == tb and np.array_equal(Ja, Jb)
    assert all(np.array_equal(la[k], lb[k]) for k in la)
    t0 = oracle.tts_eval(L, J0, betas, 4, cfg["seed"], 0, 256, 1, 1)[0]
    cur = t0
    J = J0.copy()
    for a in range(12):
        if la["accept"][a]:
            assert la["tts"][a] > cur                       # greedy: strictly harder
            cur = la["tts"][a]
            J[la["edge"][a]] = la["new"][a]
        assert la["old"][a] != la["new"][a]
    assert cur == ta and np.array_equal(J, Ja) and ta >= t0
    # split run (resume from the logged state) equals the straight run
    J1, t1, _ = oracle.engineer_run(L, J0, betas, 4, cfg["seed"], 0, 256, 1, 1, 1, 5)
    J2, t2, _ = oracle.engineer_run(L, J1, betas, 4, cfg["seed"], 0, 256, 1, 1, 6, 7, tts_cur=t1)
    assert t2 == ta and np.array_equal(J2, Ja)


# --------------------------------------------------------------------------
# Records (best energy, first sweep reaching it) against a per-sweep trace.
# --------------------------------------------------------------------------
def test_best_first_records_match_min_energy_trace():
    """first[r] must be the EARLIEST sweep whose lowest replica energy equals
    the run's final best (0 if the initial state already holds it).  The trace
    is built by stepping the oracle one sweep at a time; an exchange permutes
    energies, so the per-sweep minimum is read after it.  The instance is cold
    enough that the best is revisited many times, so recording the last hit
    instead of the first fails."""
    L, R, n = 2, 6, 300
    J = W.random_couplers(L, 91, 0)
    betas = W.beta_ladder(6, 0.3, 3.0)
    straight = oracle.PTState(L, J, betas, R, seed=91, uid=3)
    straight.sweeps(n, 1)
    stepped = oracle.PTState(L, J, betas, R, seed=91, uid=3)
    trace = [stepped.E.min(axis=1).copy()]
    for _ in range(n):
        stepped.sweeps(1, 1)
        trace.append(stepped.E.min(axis=1).copy())
    trace = np.array(trace)                                   # [n+1, R]; row s = after sweep s
    revisits = 0
    for r in range(R):
        best = trace[:, r].min()
        hits = np.flatnonzero(trace[:, r] == best)
        assert straight.best[r] == best
        assert straight.first[r] == hits[0]
        revisits += len(hits) > 1 and hits[-1] != hits[0]
    assert revisits == R                                      # every run revisits its best


# --------------------------------------------------------------------------
# Algorithm 1's acceptance: greedy, Boltzmann branch, reversed direction.
# --------------------------------------------------------------------------
def test_rao_accept_greedy_and_reversed():
    for direction in (1, -1):
        for cur, new in ((100, 101), (100, 99), (100, 100), (513, 2**16 + 1)):
            want = direction * (new - cur) > 0          # strictly better in the chosen direction
            for u in (0, 2**31, 2**32 - 1):
                assert oracle.rao_accept(cur, new, direction, -1.0, u) == want


@pytest.mark.parametrize("direction", [1, -1])
def test_rao_boltzmann_branch_frequency(direction):
    """A move that does not improve TTS is kept with probability
    exp(-beta |dTTS|) (Algorithm 1).  The uniforms are word 3 of the proposal
    draws of consecutive steps, as in the engineering loop; over n steps the
    kept fraction must lie within 5 standard errors of the exact value."""
    L = 4
    J = W.random_couplers(L, 83, 0)
    n = 20000
    us = [oracle.engineer_draw(L, J, 83, 0, t)[3] for t in range(n)]
    beta = 0.01
    for dtts in (30, 120, 400):
        p = math.exp(-beta * dtts)
        cur = 1000
        new = cur - direction * dtts                   # worse by dtts in the chosen direction
        kept = sum(oracle.rao_accept(cur, new, direction, beta, u) for u in us)
        assert abs(kept / n - p) <= 5 * math.sqrt(p * (1 - p) / n), (dtts, kept / n, p)
        # the improving move is always kept, whatever the uniform
        assert all(oracle.rao_accept(cur, cur + direction * dtts, direction, beta, u) for u in us[:200])
    # a tie has dTTS = 0: probability exp(0) = 1 keeps it under the Boltzmann rule
    assert all(oracle.rao_accept(500, 500, direction, beta, u) for u in us[:200] if u != 2**32 - 1)


def test_engineer_run_decisions_follow_rule():
    """Every logged decision of a Boltzmann, reversed RAO run equals the
    pinned acceptance rule applied to the logged TTS values and the step's
    uniform (word 3 of its proposal draw)."""
    L = 4
    J0 = W.random_couplers(L, 85, 0)
    betas = W.beta_ladder(8, 0.1, 3.0)
    S, R, seed, base = 128, 4, 85, 0
    beta_rao = 0.02
    Jf, tf, log = oracle.engineer_run(L, J0, betas, R, seed, base, S, 1, 1, 0, 16, beta_rao=beta_rao, direction=-1)
    cur = oracle.tts_eval(L, J0, betas, R, seed, base, S, 1, 1)[0]
    J = J0.copy()
    n_boltzmann = 0
    for a in range(16):
        e, v, _, u = oracle.engineer_draw(L, J, seed, base, a)
        assert (e, v) == (log["edge"][a], log["new"][a])
        want = oracle.rao_accept(cur, log["tts"][a], -1, beta_rao, u)
        assert bool(log["accept"][a]) == want
        n_boltzmann += want and log["tts"][a] >= cur
        if want:
            cur = log["tts"][a]
            J[e] = v
    assert cur == tf and np.array_equal(J, Jf)
    assert n_boltzmann >= 1                          # the Boltzmann branch was taken at least once


# --------------------------------------------------------------------------
# Proposal draws: coupler uniform over the edges, new value uniform over the
# five values other than the current one (chi-square at a fixed seed).
# --------------------------------------------------------------------------
def test_engineer_draws_uniform():
    from scipy.stats import chi2
    L = 4
    J = W.random_couplers(L, 87, 0)
    E = len(J)
    n = 60000
    edges = np.zeros(E, np.int64)
    ranks = np.zeros(5, np.int64)
    for t in range(n):
        e, v, _, _ = oracle.engineer_draw(L, J, 87, 0, t, proposal=t % 7)
        allowed = [x for x in (-3, -2, -1, 1, 2, 3) if x != J[e]]
        assert v in allowed
        edges[e] += 1
        ranks[allowed.index(v)] += 1
    def stat(c):
        exp = c.sum() / len(c)
        return float(((c - exp) ** 2 / exp).sum())
    assert stat(ranks) < chi2.ppf(0.999, 4), ranks
    assert stat(edges) < chi2.ppf(0.999, E - 1)
    # a biased draw (mulhi over 6 values, the current one skipped by moving up)
    # puts twice the mass on one value and is caught by the same bound
    biased = ranks.copy()
    biased[0] += ranks[0]
    assert stat(biased) > chi2.ppf(0.999, 4)


# --------------------------------------------------------------------------
# Doubling budget (the TTS reading for the large instances): the result is
# the first level Lv in S0, 2 S0, ... Smax whose TTS against the best energy
# found within Lv sweeps is <= Lv / 4, else unsolved = Smax + 1.  Checked
# against the same runs stepped level by level and the pinned TTS statistic.
# --------------------------------------------------------------------------
def _doubling_by_levels(L, J, betas, R, seed, uid, S0, Smax):
    st = oracle.PTState(L, J, betas, R, seed=seed, uid=uid)
    lv = S0
    while True:
        st.sweeps(lv - st.sweep, 1)
        t, h, tg = oracle.tts(st.best, st.first, oracle.TARGET_BEST, lv)
        if t <= lv // 4:
            return t, h, tg, lv
        if lv >= Smax:
            return Smax + 1, h, tg, lv
        lv *= 2


@pytest.mark.parametrize("L,NT,R,S0,Smax,seed", [(2, 4, 4, 4, 64, 93), (4, 8, 6, 8, 512, 93)])
def test_doubling_budget_matches_levels(L, NT, R, S0, Smax, seed):
    J = W.random_couplers(L, seed, 1 if L == 2 else 0)
    betas = W.beta_ladder(NT, 0.5 if L == 2 else 0.1, 3.0)
    levels = set()
    for uid in range(6):
        got = oracle.tts_eval_doubling(L, J, betas, R, seed, uid, S0, Smax, 1)
        assert got == _doubling_by_levels(L, J, betas, R, seed, uid, S0, Smax)
        levels.add((got[3], got[0] > Smax))
    assert len(levels) >= 2                    # the cases decide at different levels / outcomes
    # a single level (Smax = S0) is the plain pass of S0 sweeps with the 4x rule applied to it
    t, h, tg, lv = oracle.tts_eval_doubling(L, J, betas, R, seed, 0, S0, S0, 1)
    t1, h1, tg1 = oracle.tts_eval(L, J, betas, R, seed, 0, S0, 1, 1)
    assert (h, tg, lv) == (h1, tg1, S0) and t == (t1 if t1 <= S0 // 4 else S0 + 1)


def test_engineer_run_with_doubling_budget_replays():
    """Every logged candidate TTS is the doubling evaluation of that candidate
    under its own PT key, and the decisions follow the greedy rule."""
    L, seed, base = 2, 95, 0
    J0 = W.random_couplers(L, seed, 0)
    betas = W.beta_ladder(4, 0.5, 3.0)
    S0, Smax, R = 4, 128, 4
    Jf, tf, log = oracle.engineer_run(L, J0, betas, R, seed, base, S0, 1, 1, 0, 10, max_sweeps=Smax)
    cur = oracle.tts_eval_doubling(L, J0, betas, R, seed, base, S0, Smax)[0]
    J = J0.copy()
    for a in range(10):
        e, v, cu, _ = oracle.engineer_draw(L, J, seed, base, a)
        Jc = J.copy()
        Jc[e] = v
        assert log["tts"][a] == oracle.tts_eval_doubling(L, Jc, betas, R, seed, cu, S0, Smax)[0]
        assert bool(log["accept"][a]) == (log["tts"][a] > cur)
        if log["accept"][a]:
            J, cur = Jc, log["tts"][a]
    assert cur == tf and np.array_equal(J, Jf)
    # without a budget the same entry point is the fixed-pass loop
    a = oracle.engineer_run(L, J0, betas, R, seed, base, 16, 2, 1, 0, 4)
    b = oracle.engineer_run(L, J0, betas, R, seed, base, 16, 2, 1, 0, 4, max_sweeps=0)
    assert a[1] == b[1] and all(np.array_equal(a[2][k], b[2][k]) for k in a[2])


# --------------------------------------------------------------------------
# Appendix B's adaptive budget, in runs and sweeps.
# --------------------------------------------------------------------------
def test_adaptive_budget_rule():
    """The run count halves after every step whose cost (runs x sweeps used)
    exceeds the cap, never below n_min; the Boltzmann beta follows 6.5 n; an
    evaluation with n runs is the first n runs of a full evaluation (each
    run's streams are keyed by its own index)."""
    L, seed, base = 2, 101, 0
    J0 = W.random_couplers(L, seed, 0)
    betas = W.beta_ladder(4, 0.5, 3.0)
    S, pm, n0, nmin = 16, 2, 32, 4
    cost_max = 20 * S * pm                 # exceeded while n > 20
    t0 = oracle.tts_eval(L, J0, betas, n0, seed, base, S, pm, 1)[0]
    Jf, tf, n_after, log = oracle.engineer_run_adaptive(L, J0, betas, seed, base, S, pm, 1, 0, 8, n0, nmin, cost_max,
                                                        t0, beta_per_run=0.05)
    assert list(log["n"]) == [32, 16, 16, 16, 16, 16, 16, 16] and n_after == 16
    assert np.all(log["level"] == S * pm)
    Jf2, _, n2, log2 = oracle.engineer_run_adaptive(L, J0, betas, seed, base, S, pm, 1, 0, 8, n0, nmin, 1, t0,
                                                    beta_per_run=0.05)
    assert list(log2["n"]) == [32, 16, 8, 4, 4, 4, 4, 4] and n2 == 4
    # replay: every step's TTS is an n-run evaluation and the rule uses beta = 0.05 n
    cur, J = t0, J0.copy()
    for a in range(8):
        e, v, cu, u = oracle.engineer_draw(L, J, seed, base, a)
        Jc = J.copy()
        Jc[e] = v
        n = int(log2["n"][a])
        tn = oracle.tts_eval(L, Jc, betas, n, seed, cu, S, pm, 1)[0]
        assert tn == log2["tts"][a]
        st = oracle.PTState(L, Jc, betas, 32, seed, cu)      # first n of 32 runs: same trajectories
        st.sweeps(S * pm, 1)
        assert oracle.tts(st.best[:n], st.first[:n], oracle.TARGET_BEST, S)[0] == tn
        acc = oracle.rao_accept(cur, tn, 1, 0.05 * n, u)
        assert bool(log2["accept"][a]) == acc
        if acc:
            cur, J = tn, Jc
    assert cur == oracle.engineer_run_adaptive(L, J0, betas, seed, base, S, pm, 1, 0, 8, n0, nmin, 1, t0,
                                               beta_per_run=0.05)[1]
    assert np.array_equal(J, Jf2)
