"""Doubling sweep budget and the plain best-of-k step on the GPU vs the oracle.

The doubling budget (levels S0, 2 S0, ... Smax on the same runs; the first
level with TTS <= level / 4 decides; unsolved = Smax + 1) is compared
bit-exactly with the oracle's or_tts_eval_doubling, alone and inside the
engineering loop (Algorithm 1).  At the C_16 / 48-temperature shape, where
the oracle is too slow, the result is checked by a property that holds at any
size: the deciding level's TTS is the TTS of one plain pass of that many
sweeps on the same random streams.
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


CASES = [(2, 4, 4, 4, 64, 93, 0.5), (4, 8, 6, 8, 512, 93, 0.1), (4, 16, 8, 16, 256, 97, 0.1)]


@pytest.mark.parametrize("L,NT,R,S0,Smax,seed,bmin", CASES)
@pytest.mark.parametrize("mapping", [None, (8, 4, 1)])
def test_tts_eval_doubling_matches_oracle(P, L, NT, R, S0, Smax, seed, bmin, mapping):
    J = W.random_couplers(L, seed, 1)
    betas = W.beta_ladder(NT, bmin, 3.0)
    seen = set()
    with P.PTHandle(L, J, betas, R, seed, 0) as h:
        if mapping:
            h.set_mapping(*mapping)
        for uid in range(5):
            got = h.tts_eval_doubling(uid, S0, Smax, 1)
            want = oracle.tts_eval_doubling(L, J, betas, R, seed, uid, S0, Smax, 1)
            assert got == want, (uid, got, want)
            seen.add(got[3])
    assert len(seen) >= 1


def test_doubling_rejects_bad_budget(P):
    J = W.random_couplers(2, 1, 0)
    with P.PTHandle(2, J, W.beta_ladder(4, 0.5, 3.0), 2, 1, 0) as h:
        for S0, Smax in ((8, 12), (8, 4), (0, 8)):
            with pytest.raises(P.PTError):
                h.tts_eval_doubling(0, S0, Smax)
        with pytest.raises(P.PTError):
            h.engineer_begin(S=8, pass_mult=2, max_sweeps=64)


@pytest.mark.parametrize("spec", [1, 4])
def test_engineer_run_doubling_matches_oracle(P, spec):
    L, seed, base, S0, Smax, R = 2, 95, 0, 4, 128, 4
    J0 = W.random_couplers(L, seed, 0)
    betas = W.beta_ladder(4, 0.5, 3.0)
    Jf, tf, log = oracle.engineer_run(L, J0, betas, R, seed, base, S0, 1, 1, 0, 10, max_sweeps=Smax)
    with P.PTHandle(L, J0, betas, R, seed, base) as h:
        t0 = h.engineer_begin(S=S0, pass_mult=1, exchange_every=1, base_uid=base, max_sweeps=Smax)
        assert t0 == oracle.tts_eval_doubling(L, J0, betas, R, seed, base, S0, Smax)[0]
        res = h.engineer_run(0, 10, spec)
        assert list(res["tts_new"]) == list(log["tts"])
        assert list(res["accepted"]) == list(log["accept"])
        assert h.engineer_tts() == tf and np.array_equal(h.couplers(), Jf)
        assert h.engineer_state()[0] == tf


@pytest.mark.parametrize("max_sweeps", [0, 256])
def test_plain_best_of_k_matches_oracle(P, max_sweeps):
    """engineer_guided_step without a model evaluates proposals 0..k-1 and keeps
    the largest TTS (ties: lower index) if it beats the current one: the plain
    loop under the guided step's acceptance rule."""
    L, NT, R, seed, uid, S0 = 4, 8, 4, 20160515, 3, 32
    J = W.random_couplers(L, seed, uid)
    betas = W.beta_ladder(NT, 0.1, 3.0)

    def ev(Jc, key):
        if max_sweeps:
            return oracle.tts_eval_doubling(L, Jc, betas, R, seed, key, S0, max_sweeps)[0]
        return oracle.tts_eval(L, Jc, betas, R, seed, key, S0, 2, 1)[0]

    with P.PTHandle(L, J, betas, R, seed, uid) as h:
        tcur = h.engineer_begin(S=S0, pass_mult=1 if max_sweeps else 2, exchange_every=1, base_uid=uid,
                                max_sweeps=max_sweeps)
        assert tcur == ev(J, uid)
        Jcur, kept = J.copy(), 0
        for step in range(4):
            res, pred, ranked = h.engineer_guided_step(None, step, n_prop=16, top=4)
            assert list(ranked) == [0, 1, 2, 3] and np.all(pred == 0)
            tts = []
            for j in range(4):
                e, v, cu, _ = oracle.engineer_draw(L, Jcur, seed, uid, step, j)
                Jc = Jcur.copy()
                Jc[e] = v
                tts.append((ev(Jc, cu), Jc))
                assert res["edge"][j] == e and res["new_value"][j] == v
            assert list(res["tts_new"]) == [t for t, _ in tts]
            best = max(range(4), key=lambda j: (tts[j][0], -j))
            keep = tts[best][0] > tcur
            assert list(res["accepted"]) == [1 if (keep and j == best) else 0 for j in range(4)]
            if keep:
                Jcur, tcur = tts[best][1], tts[best][0]
                kept += 1
            assert h.engineer_tts() == tcur and np.array_equal(h.couplers(), Jcur)


def test_doubling_prefix_property_at_c16(P):
    """Config-5 shape (C_16, 48 temperatures in [0.05, 5], 32 runs): whatever
    level decides, its TTS, hits and target equal those of one plain pass of
    that many sweeps keyed by the same uid."""
    cfg = W.CONFIGS["c16_guided"]
    J = W.random_couplers(16, cfg["seed"], 0)
    betas = W.beta_ladder(cfg["n_temps"], cfg["beta_min"], cfg["beta_max"])
    S0, Smax = 256, 4096
    with P.PTHandle(16, J, betas, cfg["n_runs"], cfg["seed"], 0) as h:
        for uid in (0, 1):
            t, hits, tg, lv = h.tts_eval_doubling(uid, S0, Smax)
            assert lv in (256, 512, 1024, 2048, 4096)
            tp, hp, tgp = h.tts_eval(uid, lv, 1, 1)
            assert (hits, tg) == (hp, tgp)
            assert t == (tp if tp <= lv // 4 else Smax + 1)
            if t <= Smax:
                assert t <= lv // 4


@pytest.mark.parametrize("max_sweeps", [0, 256])
def test_tts_eval_many_matches_oracle(P, max_sweeps):
    """Batched evaluation of unrelated coupler vectors, each under its own key."""
    L, NT, R, seed, S0 = 4, 8, 4, 99, 16
    betas = W.beta_ladder(NT, 0.1, 3.0)
    Js = np.stack([W.random_couplers(L, seed, i) for i in range(6)])
    uids = [7, 3, 3, 100, 2**32 - 1, 12]
    with P.PTHandle(L, Js[0], betas, R, seed, 0) as h:
        out = h.tts_eval_many(Js, uids, S0, 1 if max_sweeps else 4, max_sweeps)
    for j in range(6):
        if max_sweeps:
            want = oracle.tts_eval_doubling(L, Js[j], betas, R, seed, uids[j], S0, max_sweeps)
        else:
            want = oracle.tts_eval(L, Js[j], betas, R, seed, uids[j], S0, 4, 1) + (4 * S0,)
        got = tuple(int(out[k][j]) for k in ("tts", "n_hit", "target", "level"))
        assert got == want, (j, got, want)


def test_engineer_run_step_log(P, tmp_path):
    """Per-step JSON records of engineer_run and lao_run match the returned results."""
    import json
    L, NT, R, seed = 2, 4, 4, 95
    J0 = W.random_couplers(L, seed, 0)
    betas = W.beta_ladder(NT, 0.5, 3.0)
    path = tmp_path / "steps.jsonl"
    with P.PTHandle(L, J0, betas, R, seed, 0) as h:
        h.engineer_begin(S=8, pass_mult=1, max_sweeps=64)
        res = h.engineer_run(0, 6, 3, log=str(path))
        recs = [json.loads(x) for x in path.read_text().splitlines()]
        assert [r["step"] for r in recs] == list(range(6))
        for i, r in enumerate(recs):
            assert (r["coupler"], r["J_old"], r["J_new"], r["tts_new"], r["accepted"]) == (
                res["edge"][i], res["old_value"][i], res["new_value"][i], res["tts_new"][i], bool(res["accepted"][i]))
            assert r["device_ms_per_eval"] > 0
        assert recs[-1]["n_hit_now"] == h.engineer_state()[1]
        h.lao_begin(64, 3, 6, 5)
        with open(path, "a") as f:
            lres = h.lao_run(1, 4, 2, log=f)
    recs = [json.loads(x) for x in path.read_text().splitlines()][6:]
    assert [r["kind"] for r in recs] == ["lao"] * 4
    assert [r["removed_loop"] for r in recs] == list(lres["removed"])


@pytest.mark.parametrize("spec,max_sweeps", [(1, 0), (4, 0), (4, 64)])
def test_adaptive_budget_matches_oracle(P, spec, max_sweeps):
    """Appendix B's rule in runs and sweeps: the run count of every step, its
    TTS and decision, and the halvings equal the oracle's; speculative
    batches are cut where the run count changes."""
    L, seed, base, NT = 2, 101, 0, 4
    J0 = W.random_couplers(L, seed, 0)
    betas = W.beta_ladder(NT, 0.5, 3.0)
    S, pm, n0, nmin = (16, 2, 32, 4) if not max_sweeps else (8, 1, 32, 4)
    cost_max = 10 * S * pm if not max_sweeps else 12 * 16
    with P.PTHandle(L, J0, betas, n0, seed, base) as h:
        t0 = h.engineer_begin(S=S, pass_mult=pm, base_uid=base, max_sweeps=max_sweeps)
        h.set_adaptive(n0, nmin, cost_max, beta_per_run=0.05)
        res = h.engineer_run(0, 10, spec)
        n_after = h.adaptive_runs()
        J_gpu, t_gpu = h.couplers(), h.engineer_tts()
    Jf, tf, n2, log = oracle.engineer_run_adaptive(L, J0, betas, seed, base, S, pm, 1, 0, 10, n0, nmin, cost_max, t0,
                                                   beta_per_run=0.05, max_sweeps=max_sweeps)
    assert list(res["n_runs"]) == list(log["n"]) and list(res["level"]) == list(log["level"])
    assert list(res["tts_new"]) == list(log["tts"]) and list(res["accepted"]) == list(log["accept"])
    assert n_after == n2 and t_gpu == tf and np.array_equal(J_gpu, Jf)
    assert len(set(log["n"])) >= 2                    # the run count did change


def _split_run(h, step0, lengths, spec):
    """engineer_run over consecutive calls of the given lengths; results concatenated."""
    parts, step = [], step0
    for n in lengths:
        parts.append(h.engineer_run(step, n, spec))
        step += n
    return {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}


@pytest.mark.parametrize("beta_rao,direction", [(-1.0, 1), (0.02, 1), (-1.0, -1)])
def test_engineer_run_split_calls_match_one_call_and_oracle(P, beta_rao, direction):
    """Each speculative batch is evaluated in full and the candidates past a
    call's end are kept for the next call: splitting 30 steps into calls of
    3, 5, 1, 7, 8, 6 with speculation 8 gives every decision of one 30-step
    call with speculation 1 and of the oracle's sequential loop."""
    L, NT, R, S, seed = 4, 8, 4, 128, 51
    J = W.random_couplers(L, seed, 0)
    betas = W.beta_ladder(NT, 0.1, 3.0)
    out = []
    for lengths, spec in (([30], 1), ([3, 5, 1, 7, 8, 6], 8), ([16, 14], 16)):
        with P.PTHandle(L, J, betas, R, seed, 0) as h:
            h.engineer_begin(S=S, pass_mult=2, exchange_every=1, base_uid=0, beta_rao=beta_rao, direction=direction)
            r = _split_run(h, 0, lengths, spec)
            out.append((r, h.engineer_tts(), h.couplers()))
    for r, t, Jc in out[1:]:
        assert all(np.array_equal(r[k], out[0][0][k]) for k in r)
        assert t == out[0][1] and np.array_equal(Jc, out[0][2])
    Jo, to, lo = oracle.engineer_run(L, J, betas, R, seed, 0, S, 2, 1, 0, 30, beta_rao=beta_rao, direction=direction)
    assert list(out[0][0]["accepted"]) == list(lo["accept"]) and out[0][1] == to and np.array_equal(out[0][2], Jo)


def test_engineer_run_kept_candidates_dropped_on_coupler_change(P):
    """A coupler set between two calls drops the candidates the first call
    evaluated past its end: the second call equals a fresh loop from the new
    couplers (same TTS baseline), not the kept evaluations."""
    L, NT, R, S, seed = 4, 8, 4, 128, 53
    J = W.random_couplers(L, seed, 0)
    betas = W.beta_ladder(NT, 0.1, 3.0)
    with P.PTHandle(L, J, betas, R, seed, 0) as h:
        h.engineer_begin(S=S, pass_mult=2, exchange_every=1, base_uid=0)
        h.engineer_run(0, 2, 8)                      # evaluates steps 0..7, keeps those past step 1
        Jm = h.couplers().copy()
        Jm[5] = -Jm[5]
        h.set_coupler(5, int(Jm[5]))
        tts = h.engineer_tts()
        r = h.engineer_run(2, 6, 8)
        got = (r, h.engineer_tts(), h.couplers())
    Jo, to, lo = oracle.engineer_run(L, Jm, betas, R, seed, 0, S, 2, 1, 2, 6, tts_cur=tts)
    assert list(got[0]["accepted"]) == list(lo["accept"]) and got[1] == to and np.array_equal(got[2], Jo)


def test_adaptive_budget_split_calls_match_oracle(P):
    """The adaptive budget with calls of 2, 3, 5 steps at speculation 4: run
    counts, TTS values, decisions and halvings equal the oracle's."""
    L, seed, base, NT = 2, 101, 0, 4
    J0 = W.random_couplers(L, seed, 0)
    betas = W.beta_ladder(NT, 0.5, 3.0)
    S, pm, n0, nmin = 16, 2, 32, 4
    cost_max = 10 * S * pm
    with P.PTHandle(L, J0, betas, n0, seed, base) as h:
        t0 = h.engineer_begin(S=S, pass_mult=pm, base_uid=base)
        h.set_adaptive(n0, nmin, cost_max, beta_per_run=0.05)
        res = _split_run(h, 0, [2, 3, 5], 4)
        n_after = h.adaptive_runs()
        J_gpu, t_gpu = h.couplers(), h.engineer_tts()
    Jf, tf, n2, log = oracle.engineer_run_adaptive(L, J0, betas, seed, base, S, pm, 1, 0, 10, n0, nmin, cost_max, t0,
                                                   beta_per_run=0.05)
    assert list(res["n_runs"]) == list(log["n"]) and list(res["tts_new"]) == list(log["tts"])
    assert list(res["accepted"]) == list(log["accept"])
    assert n_after == n2 and t_gpu == tf and np.array_equal(J_gpu, Jf)
