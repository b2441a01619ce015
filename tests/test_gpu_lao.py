"""Loop adaptive optimisation (Algorithm 2) on the GPU against the oracle:
planted instance, known-target TTS of every candidate, and every decision,
bit-exact; speculative batches give the step-by-step results."""
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


@pytest.mark.parametrize("L,NT,R,M,S,beta,spec,w", [(2, 6, 4, 10, 128, -1.0, 1, 3), (4, 8, 8, 40, 256, 0.05, 4, 3),
                                                    (4, 8, 8, 40, 256, -1.0, 16, 3), (2, 6, 4, 10, 128, -1.0, 1, 5),
                                                    (4, 8, 8, 60, 256, 0.05, 4, 5), (4, 8, 8, 60, 256, -1.0, 16, 5)])
def test_lao_matches_oracle(P, L, NT, R, M, S, beta, spec, w):
    """Weights 1..w (the paper's [1, 5]); couplers of overlapping loops sum past
    +-3, so the handle's Metropolis table grows beyond 19 rows."""
    seed, uid, steps = 20160516, 21, 14
    betas = W.beta_ladder(NT, 0.1, 3.0)
    ref = oracle.LAOState(L, betas, R, seed, uid, M, w_max=w, S=S, beta_rao=beta)
    log = ref.run(1, steps)
    with P.PTHandle(L, np.zeros(W.chimera_n_edges(L), np.int8), betas, R, seed, 0) as h:
        t0 = h.lao_begin(S, uid, M, w, 1, beta)
        res = h.lao_run(1, steps, spec)
        st = h.lao_state()
        rows = h.table_rows()
    assert np.array_equal(res["removed"], log["removed"])
    assert np.array_equal(res["tts_new"], log["tts"])
    assert np.array_equal(res["E_gs_new"], log["E_gs"])
    assert np.array_equal(res["accepted"], log["accepted"])
    assert np.array_equal(st["loops"], ref.loops) and np.array_equal(st["J"], ref.J)
    assert st["E_gs"] == ref.E_gs and st["tts"] == ref.tts
    assert t0 == res["tts_old"][0]
    assert oracle.energy(L, st["J"], st["planted"]) == st["E_gs"]
    if w == 5 and L == 4:
        assert np.abs(st["J"]).max() > 3 and rows > 19


def test_lao_c8_shape_known_target(P):
    """C_8 with 350 loops: the planted energy is a lower bound every run respects,
    and runs that reach it count as hits (a short pass, properties only)."""
    cfg = W.CONFIGS["c8_single"]
    betas = W.beta_ladder(cfg["n_temps"], cfg["beta_min"], cfg["beta_max"])
    with P.PTHandle(8, np.zeros(W.chimera_n_edges(8), np.int8), betas, cfg["n_runs"], cfg["seed"], 0) as h:
        h.lao_begin(1 << 12, 7, 350, 5)
        st = h.lao_state()
        h.reset(0)                                   # fresh runs on the planted couplers
        h.sweep(512, 1)
        s = h.state()
        assert np.all(s["best"] >= st["E_gs"]) and np.all(s["E"] >= st["E_gs"])
        tts, nhit, target = h.tts(st["E_gs"], 512)
        assert target == st["E_gs"] and 0 <= nhit <= cfg["n_runs"]


@pytest.mark.parametrize("planted", [True, False])
def test_overlaps_match_oracle(P, planted):
    """Ground / first-excited overlaps of the runs' replicas (pairwise distances
    on the GPU) against the oracle's definition."""
    L, NT, R, seed = 4, 16, 32, 20160517
    betas = W.beta_ladder(NT, 0.1, 3.0)
    if planted:
        _, _, J, E_gs = oracle.lao_plant(L, seed, 3, 40)
    else:
        J, E_gs = W.random_couplers(L, seed, 3), None
    with P.PTHandle(L, J, betas, R, seed, 5) as h:
        h.sweep(1500, 1)
        st = h.state()
        if E_gs is None:
            E_gs = int(st["best"].min())
        r = h.overlaps(E_gs)
    ref = oracle.overlaps(st["spins"], st["E"], E_gs)
    assert r == ref
    assert r["n_gs"] >= 1 and r["n_es"] >= 1


@pytest.mark.parametrize("beta,spec,lengths", [(-1.0, 8, [3, 5, 1, 5]), (0.05, 16, [7, 7])])
def test_lao_split_calls_match_oracle(P, beta, spec, lengths):
    """lao_run evaluates every batch in full and keeps the evaluations past a
    call's end for the next call: uneven calls give the oracle's decisions,
    loops, couplers and E_GS."""
    L, NT, R, M, S, w = 4, 8, 8, 40, 256, 5
    seed, uid, steps = 20160516, 23, sum(lengths)
    betas = W.beta_ladder(NT, 0.1, 3.0)
    ref = oracle.LAOState(L, betas, R, seed, uid, M, w_max=w, S=S, beta_rao=beta)
    log = ref.run(1, steps)
    with P.PTHandle(L, np.zeros(W.chimera_n_edges(L), np.int8), betas, R, seed, 0) as h:
        h.lao_begin(S, uid, M, w, 1, beta)
        parts, step = [], 1
        for n in lengths:
            parts.append(h.lao_run(step, n, spec))
            step += n
        st = h.lao_state()
    res = {k: np.concatenate([p[k] for p in parts]) for k in ("removed", "tts_new", "E_gs_new", "accepted")}
    assert np.array_equal(res["removed"], log["removed"]) and np.array_equal(res["tts_new"], log["tts"])
    assert np.array_equal(res["E_gs_new"], log["E_gs"]) and np.array_equal(res["accepted"], log["accepted"])
    assert np.array_equal(st["loops"], ref.loops) and np.array_equal(st["J"], ref.J)
    assert st["E_gs"] == ref.E_gs and st["tts"] == ref.tts
