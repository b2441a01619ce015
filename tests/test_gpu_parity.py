"""GPU path vs the CPU oracle, element by element, through the C ABI.

Spins, energies, slot maps, best/first records, acceptance counters, TTS and
engineering decisions must match bit-exactly (integer work: no tolerance).
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1605_03607_gb300 as pkg
    from paper_1605_03607_gb300 import build as b
    b.build()
    pkg.load()
    return pkg


def _assert_state_equal(st, ref, ctx=""):
    assert st["sweep"] == ref.sweep, ctx
    for k in ("spins", "E", "best", "first", "macc"):
        a, b = st[k], getattr(ref, k)
        if not np.array_equal(a, b):
            bad = np.argwhere(a != b)
            raise AssertionError(f"{ctx}: {k} differs at {bad[:5].tolist()} ({len(bad)} entries)")
    if ref.NT > 1:
        assert np.array_equal(st["xacc"], ref.xacc), f"{ctx}: xacc"


def _pair(P, L, NT, R, seed=7, uid=3, bmin=0.1, bmax=3.0, J=None):
    J = W.random_couplers(L, seed, uid) if J is None else J
    betas = W.beta_ladder(NT, bmin, bmax)
    return P.PTHandle(L, J, betas, R, seed, uid), oracle.PTState(L, J, betas, R, seed, uid), J, betas


# ---------------------------------------------------------------------------
def test_tables_equal_oracle(P):
    for NT, lo, hi in ((16, 0.1, 3.0), (32, 0.1, 4.0), (48, 0.05, 5.0), (2, 0.5, 0.6)):
        h, _, _, betas = _pair(P, 4, NT, 1, bmin=lo, bmax=hi)
        thr, xoff, xthr = h.tables()
        othr = oracle.metropolis_thresholds(betas)
        assert np.array_equal(thr[:, 1:], othr[:, 1:])
        ooff, otab = oracle.exchange_thresholds(betas)
        assert np.array_equal(xoff[:NT - 1], ooff[:NT - 1]) and np.array_equal(xthr, otab)
        h.close()


def test_initial_state(P):
    h, ref, _, _ = _pair(P, 4, 16, 8)
    _assert_state_equal(h.state(), ref, "init")
    assert np.all(h.state()["perm"] == np.arange(16))


SHAPES = [
    # L, NT, R, sweeps, exchange_every, schedule (slot_parallel, runs_per_cta, sweeps_per_launch)
    (4, 16, 8, 200, 1, None),
    (4, 16, 8, 200, 1, (2, 4, 0)),
    (4, 16, 5, 120, 3, (4, 3, 0)),              # ragged runs per CTA
    (4, 16, 8, 150, 1, (16, 2, 7)),             # many launches of 7 sweeps
    (8, 32, 4, 60, 1, None),
    (8, 32, 3, 60, 1, (1, 2, 0)),
    (8, 32, 3, 40, 2, (16, 1, 0)),              # 1024 threads per run
    (12, 24, 2, 20, 1, None),
    (16, 48, 2, 8, 1, None),
    (1, 4, 3, 300, 1, None),                    # per-lane atomics (warp spans many slots)
    (2, 6, 3, 300, 1, None),
    (3, 5, 2, 100, 2, None),
    (5, 8, 2, 100, 1, None),
    (4, 1, 4, 150, 1, None),                    # one temperature: no exchange
    (4, 2, 4, 150, 1, None),
    (4, 64, 2, 40, 1, None),                    # maximum slots
    (4, 33, 3, 90, 1, None),                    # first slot count with two slots per exchange lane
]


@pytest.mark.parametrize("L,NT,R,n,x,sched", SHAPES)
def test_sweeps_bit_exact(P, L, NT, R, n, x, sched):
    h, ref, _, _ = _pair(P, L, NT, R, seed=11 + L, uid=NT)
    if sched:
        h.set_schedule(*sched)
    h.sweep(n // 2, x)
    h.sweep(n - n // 2, x)
    ref.sweeps(n // 2, x)
    ref.sweeps(n - n // 2, x)
    st = h.state()
    _assert_state_equal(st, ref, f"L={L} NT={NT} R={R} sched={sched}")
    assert np.array_equal(st["E"], ref.full_energies())
    h.close()


SLOT_MAJOR = [
    # L, NT, R, sweeps, exchange_every, (team, slot_parallel teams, runs_per_cta)
    (4, 16, 8, 150, 1, (4, 16, 1)),
    (4, 16, 5, 120, 2, (2, 16, 2)),             # ragged runs per CTA
    (8, 32, 4, 60, 1, (4, 32, 1)),
    (8, 32, 3, 60, 1, (16, 8, 2)),              # a team owns 4 slots
    (8, 32, 3, 40, 3, (32, 4, 1)),
    (12, 24, 2, 20, 1, (8, 24, 1)),
    (16, 48, 2, 8, 1, (16, 24, 1)),
    (1, 4, 3, 300, 1, (8, 4, 1)),               # more lanes than cells
    (5, 8, 2, 100, 1, (4, 8, 1)),
    (4, 1, 4, 150, 1, (32, 1, 1)),              # one temperature
    (4, 64, 2, 40, 1, (2, 64, 2)),              # maximum slots
    (4, 33, 3, 90, 1, (4, 32, 1)),              # two slots per exchange lane, 33 buffers on 32 teams
]


@pytest.mark.parametrize("L,NT,R,n,x,mapping", SLOT_MAJOR)
def test_slot_major_bit_exact(P, L, NT, R, n, x, mapping):
    h, ref, _, _ = _pair(P, L, NT, R, seed=19 + L, uid=NT + 1)
    h.set_mapping(*mapping)
    assert h.mapping() == mapping[0]
    h.sweep(n // 3, x)
    h.sweep(n - n // 3, x)
    ref.sweeps(n // 3, x)
    ref.sweeps(n - n // 3, x)
    _assert_state_equal(h.state(), ref, f"slot-major L={L} NT={NT} {mapping}")
    h.exchange()
    ref.exchange()
    _assert_state_equal(h.state(), ref, "slot-major standalone exchange")
    h.close()


def test_autotune_keeps_results(P):
    h, ref, _, _ = _pair(P, 8, 32, 4, seed=3, uid=3)
    h.autotune(n_inst=4, trial_sweeps=8)
    h.sweep(50, 1)
    ref.sweeps(50, 1)
    _assert_state_equal(h.state(), ref, f"autotuned {h.schedule()} team {h.mapping()}")


def test_schedule_and_split_invariance(P):
    outs = []
    for sched in ((0, 0, 4096), (2, 1, 1), (8, 4, 13), (16, 4, 64)):
        h, _, _, _ = _pair(P, 4, 16, 8, seed=5, uid=9)
        h.set_schedule(*sched)
        h.sweep(97, 1)
        outs.append(h.state())
        h.close()
    for o in outs[1:]:
        for k in ("spins", "E", "perm", "best", "first", "macc", "xacc"):
            assert np.array_equal(o[k], outs[0][k]), k


def test_standalone_exchange(P):
    h, ref, _, _ = _pair(P, 4, 12, 4, seed=17, uid=1)
    for _ in range(15):
        h.sweep(3, 0)
        h.exchange()
        ref.sweeps(3, 0)
        ref.exchange()
    _assert_state_equal(h.state(), ref, "standalone exchange")


def test_narrow_ladder_exchange_bit_exact(P):
    """Close temperatures (64 slots in beta [0.30, 0.35]) make exchange tables of
    about 15,000 entries per pair, so the critical gaps reach the thousands and
    the float estimate of each gap carries its largest absolute error.  Every
    exchange decision must still equal the oracle's table search, in both
    mappings."""
    for mapping in (None, (2, 64, 2)):
        h, ref, _, _ = _pair(P, 2, 64, 4, seed=31, uid=5, bmin=0.30, bmax=0.35)
        if mapping:
            h.set_mapping(*mapping)
        h.sweep(300, 1)
        ref.sweeps(300, 1)
        _assert_state_equal(h.state(), ref, f"narrow ladder, mapping {mapping}")
        assert ref.xacc.sum() > 0
        h.close()


def test_set_spins_and_gauge(P):
    L, NT, R = 4, 8, 3
    J = W.random_couplers(L, 23, 0)
    betas = W.beta_ladder(NT, 0.2, 2.5)
    ei, ej = oracle.chimera_edges(L)
    g = np.where(np.random.default_rng(4).integers(0, 2, 8 * L * L) == 0, -1, 1).astype(np.int8)
    Jg = (g[ei] * g[ej] * J).astype(np.int8)
    s0 = W.random_spins((R, NT, 8 * L * L), 99)
    a = P.PTHandle(L, J, betas, R, 23, 5)
    b = P.PTHandle(L, Jg, betas, R, 23, 5)
    a.set_spins(s0)
    b.set_spins(s0 * g)
    ref = oracle.PTState(L, J, betas, R, 23, 5, spins=s0)
    for _ in range(3):
        a.sweep(40, 1)
        b.sweep(40, 1)
        ref.sweeps(40, 1)
        sa, sb = a.state(), b.state()
        assert np.array_equal(sb["spins"], sa["spins"] * g)
        for k in ("E", "perm", "best", "first", "macc", "xacc"):
            assert np.array_equal(sa[k], sb[k]), k
        _assert_state_equal(sa, ref, "set_spins")
    with pytest.raises(P.PTError):
        a.set_spins(np.zeros((R, NT, 8 * L * L), np.int8))


def test_tts_reduction(P):
    h, ref, _, _ = _pair(P, 4, 16, 8, seed=31, uid=2)
    h.sweep(300, 1)
    ref.sweeps(300, 1)
    st = h.state()
    for target in (P.PT_TARGET_BEST, int(st["best"].min()) + 4, int(st["best"].min()) - 2):
        for horizon in (300, 150, 20, 0):
            assert h.tts(target, horizon) == oracle.tts(ref.best, ref.first, target, horizon)


@pytest.mark.parametrize("pass_mult", [1, 4])
def test_tts_eval_small(P, pass_mult):
    L, NT, R = 4, 16, 8
    J = W.random_couplers(L, 41, 0)
    betas = W.beta_ladder(NT, 0.1, 3.0)
    h = P.PTHandle(L, J, betas, R, 41, 0)
    for uid in (0, 7):
        assert h.tts_eval(uid, 256, pass_mult, 1) == oracle.tts_eval(L, J, betas, R, 41, uid, 256, pass_mult, 1)


def test_tts_eval_tiny_config_full(P):
    """The tiny configuration in full: C_4, 16 temperatures in [0.1, 3], 8 runs x 2048 sweeps."""
    cfg = W.CONFIGS["c4_tiny"]
    J = W.random_couplers(cfg["L"], cfg["seed"], 0)
    betas = W.beta_ladder(cfg["n_temps"], cfg["beta_min"], cfg["beta_max"])
    h = P.PTHandle(cfg["L"], J, betas, cfg["n_runs"], cfg["seed"], 0)
    got = h.tts_eval(0, cfg["sweeps"], cfg["pass_mult"], cfg["exchange_every"])
    want = oracle.tts_eval(cfg["L"], J, betas, cfg["n_runs"], cfg["seed"], 0, cfg["sweeps"],
                           cfg["pass_mult"], cfg["exchange_every"])
    assert got == want


def test_engineering_tiny_config(P):
    """Algorithm 1 on the tiny configuration: 20 greedy steps, speculative batches of 4."""
    cfg = W.CONFIGS["c4_tiny"]
    L, S = cfg["L"], cfg["sweeps"]
    J = W.random_couplers(L, cfg["seed"], 0)
    betas = W.beta_ladder(cfg["n_temps"], cfg["beta_min"], cfg["beta_max"])
    h = P.PTHandle(L, J, betas, cfg["n_runs"], cfg["seed"], 0)
    t0 = h.engineer_begin(S=S, pass_mult=1, exchange_every=1, base_uid=0)
    res = h.engineer_run(0, cfg["steps"], speculation=4)
    Jo, to, lo = oracle.engineer_run(L, J, betas, cfg["n_runs"], cfg["seed"], 0, S, 1, 1, 0, cfg["steps"])
    assert t0 == oracle.tts_eval(L, J, betas, cfg["n_runs"], cfg["seed"], 0, S, 1, 1)[0]
    assert list(res["edge"]) == list(lo["edge"])
    assert list(res["new_value"]) == list(lo["new"])
    assert list(res["tts_new"]) == list(lo["tts"])
    assert list(res["accepted"]) == list(lo["accept"])
    assert h.engineer_tts() == to
    assert np.array_equal(h.couplers(), Jo)


@pytest.mark.parametrize("beta_rao,direction", [(-1.0, 1), (0.02, 1), (-1.0, -1)])
def test_engineering_speculation_invariance(P, beta_rao, direction):
    L, NT, R, S = 4, 8, 4, 128
    J = W.random_couplers(L, 51, 0)
    betas = W.beta_ladder(NT, 0.1, 3.0)
    runs = []
    for spec in (1, 3, 8):
        h = P.PTHandle(L, J, betas, R, 51, 0)
        h.engineer_begin(S=S, pass_mult=2, exchange_every=1, base_uid=0, beta_rao=beta_rao, direction=direction)
        r = h.engineer_run(0, 24, speculation=spec)
        runs.append((r, h.engineer_tts(), h.couplers()))
        h.close()
    for r, t, Jc in runs[1:]:
        assert all(np.array_equal(r[k], runs[0][0][k]) for k in r)
        assert t == runs[0][1] and np.array_equal(Jc, runs[0][2])
    Jo, to, lo = oracle.engineer_run(L, J, betas, R, 51, 0, S, 2, 1, 0, 24, beta_rao=beta_rao, direction=direction)
    assert list(runs[0][0]["accepted"]) == list(lo["accept"]) and runs[0][1] == to


def test_checkpoint_resume(P):
    h, _, _, _ = _pair(P, 4, 16, 6, seed=61, uid=4)
    h.sweep(200, 1)
    straight = h.state()
    h2, _, _, _ = _pair(P, 4, 16, 6, seed=61, uid=4)
    h2.sweep(100, 1)
    buf = h2.checkpoint()
    h2.close()
    h3, _, _, _ = _pair(P, 4, 16, 6, seed=61, uid=999)
    h3.restore(buf)
    h3.sweep(100, 1)
    resumed = h3.state()
    for k in ("spins", "E", "perm", "best", "first", "macc", "xacc"):
        assert np.array_equal(straight[k], resumed[k]), k
    bad = buf.copy()
    bad[64 + 3] = 0x80                                 # a coupler byte of -128: outside [-127, 127]
    with pytest.raises(P.PTError):
        h3.restore(bad)
    bad = buf.copy()
    bad[64 + 3] = 125                                  # its spins' sums of |J| would exceed 127
    with pytest.raises(P.PTError):
        h3.restore(bad)
    with pytest.raises(P.PTError):
        h3.restore(buf[:-1])


def test_set_coupler_energies(P):
    h, ref, J, _ = _pair(P, 4, 8, 3, seed=71, uid=0)
    h.sweep(50, 1)
    h.set_coupler(17, -3)
    J2 = J.copy()
    J2[17] = -3
    st = h.state()
    want = np.array([[oracle.energy(4, J2, st["spins"][r, t]) for t in range(8)] for r in range(3)])
    assert np.array_equal(st["E"], want)
    assert np.array_equal(st["best"], want.min(axis=1)) and np.all(st["first"] == 50)
    with pytest.raises(P.PTError):
        h.set_coupler(len(J), 1)


def test_zero_sweeps_and_single_run(P):
    h, ref, _, _ = _pair(P, 4, 16, 1, seed=81, uid=0)
    h.sweep(0, 1)
    _assert_state_equal(h.state(), ref, "zero sweeps")
    h.sweep(64, 1)
    ref.sweeps(64, 1)
    _assert_state_equal(h.state(), ref, "R=1")
    assert h.tts() == ref.tts()


@pytest.mark.parametrize("mapping", [None, (4, 32, 1)])
def test_single_instance_config_launch_shape(P, mapping):
    """C_8, 32 temperatures in [0.1, 4], 64 runs, with the default schedule and
    with the one the bench's autotuner picks (slot-major, team 4, 32 teams, one
    run per CTA, 4096 sweeps per launch): a prefix compared element by element,
    then a full 4x pass checked through properties that hold at any length."""
    cfg = W.CONFIGS["c8_single"]
    L, NT, R = cfg["L"], cfg["n_temps"], cfg["n_runs"]
    J = W.random_couplers(L, cfg["seed"], 0)
    betas = W.beta_ladder(NT, cfg["beta_min"], cfg["beta_max"])
    h = P.PTHandle(L, J, betas, R, cfg["seed"], 0)
    if mapping:
        h.set_mapping(*mapping)
        h.set_schedule(0, 0, 4096)
    ref = oracle.PTState(L, J, betas, R, cfg["seed"], 0)
    h.sweep(96, 1)
    ref.sweeps(96, 1)
    _assert_state_equal(h.state(), ref, "C_8 prefix")
    tts, nhit, target = h.tts_eval(1, cfg["sweeps"], cfg["pass_mult"], 1)
    st = h.state()
    assert st["sweep"] == cfg["sweeps"] * cfg["pass_mult"]
    for r in (0, 17, 63):
        for t in (0, 15, 31):
            assert st["E"][r, t] == oracle.energy(L, J, st["spins"][r, t])
    assert np.all(st["best"] <= st["E"].min(axis=1)) and target == st["best"].min()
    assert (tts, nhit, target) == oracle.tts(st["best"], st["first"], oracle.TARGET_BEST, cfg["sweeps"])
    assert np.all(np.sort(st["perm"], axis=1) == np.arange(NT))
    assert st["macc"].sum() > 0 and st["xacc"].sum() > 0


def test_large_couplers_and_table_growth(P):
    """Couplers beyond +-3 (planted instances sum loop weights): the Metropolis
    table has one row per local-field value up to the largest sum of |J| over a
    spin's couplers.  A handle created on +-3 couplers (19 rows) whose coupler
    change needs more rows enlarges its table; fresh runs on the changed
    couplers then match the oracle bit-exactly."""
    L, NT, R, seed = 4, 8, 4, 20160518
    betas = W.beta_ladder(NT, 0.1, 3.0)
    rng = np.random.default_rng(3)
    Jbig = rng.integers(-9, 10, size=W.chimera_n_edges(L)).astype(np.int8)
    with P.PTHandle(L, Jbig, betas, R, seed, 4) as h:
        assert h.table_rows() >= oracle.coupler_kmax(L, Jbig) + 1 > 19
        h.sweep(120, 1)
        ref = oracle.PTState(L, Jbig, betas, R, seed, 4)
        ref.sweeps(120, 1)
        _assert_state_equal(h.state(), ref, "couplers in [-9, 9]")
    J = W.random_couplers(L, seed, 0)
    with P.PTHandle(L, J, betas, R, seed, 5) as h:
        assert h.table_rows() == 19
        h.set_coupler(0, 90)                 # spin 0 (and 4): sum of |J| well above 18
        J2 = J.copy()
        J2[0] = 90
        rows = h.table_rows()
        assert rows >= oracle.coupler_kmax(L, J2) + 1
        h.reset(5)
        h.sweep(80, 1)
        ref = oracle.PTState(L, J2, betas, R, seed, 5)
        ref.sweeps(80, 1)
        _assert_state_equal(h.state(), ref, "after table growth")
        with pytest.raises(P.PTError):
            h.set_coupler(1, 100)           # spin 0's sum would exceed 127
        assert h.table_rows() == rows and np.array_equal(h.couplers(), J2)


def test_graph_form_matches_full_vector(P):
    """pt_create_graph with a shuffled coupler list that omits some couplers
    (inoperative qubits, as on the paper's 504-qubit device): the handle holds
    the full C_L vector with zeros where nothing was listed, and its runs
    match the oracle on that vector bit-exactly."""
    L, NT, R, seed = 4, 8, 4, 20160520
    ei, ej = oracle.chimera_edges(L)
    J = W.random_couplers(L, seed, 0)
    rng = np.random.default_rng(9)
    dead = {int(x) for x in rng.choice(8 * L * L, 4, replace=False)}          # four inoperative spins
    keep = [e for e in range(len(J)) if int(ei[e]) not in dead and int(ej[e]) not in dead]
    order = rng.permutation(keep)
    flip = rng.random(len(order)) < 0.5                                        # either orientation
    a = np.where(flip, ej[order], ei[order])
    b = np.where(flip, ei[order], ej[order])
    full = np.zeros_like(J)
    full[keep] = J[keep]
    betas = W.beta_ladder(NT, 0.1, 3.0)
    with P.PTHandle(L, J[order], betas, R, seed, 2, edges=(a, b)) as h:
        assert np.array_equal(h.couplers(), full)
        h.sweep(100, 1)
        st = h.state()
    ref = oracle.PTState(L, full, betas, R, seed, 2)
    ref.sweeps(100, 1)
    _assert_state_equal(st, ref, "graph form")
