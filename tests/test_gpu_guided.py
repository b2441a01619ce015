"""Surrogate-guided RAO step vs the oracles.

The ranking is a floating-point decision: the GPU's predictions are checked
against the FP64 surrogate (2e-2) and the ranking against the GPU's own
predictions; given that ranking, the candidates' TTS and the kept move must
match the PT oracle bit-exactly.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import surrogate as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1605_03607_gb300 as pkg
    from paper_1605_03607_gb300 import build as b
    b.build()
    pkg.load()
    return pkg


def test_guided_step_matches_oracle(P):
    L, NT, R, seed, uid, Sw = 4, 8, 4, 20160515, 3, 128
    J = W.random_couplers(L, seed, uid)
    betas = W.beta_ladder(NT, 0.1, 3.0)
    theta = W.surrogate_init_params(5)
    with P.Surrogate() as m, P.PTHandle(L, J, betas, R, seed, uid) as h:
        m.set_params(theta)
        t0 = h.engineer_begin(S=Sw, pass_mult=2, exchange_every=1, base_uid=uid)
        Jcur, tcur = J.copy(), t0
        for step in range(3):
            res, pred, ranked = h.engineer_guided_step(m, step, n_prop=24, top=4)
            props = []
            for j in range(24):
                e, v, cu, ua = oracle.engineer_draw(L, Jcur, seed, uid, step, j)
                Jc = Jcur.copy()
                Jc[e] = v
                props.append((Jc, e, v, cu))
            ref_pred = S.forward(theta.astype(np.float32).astype(np.float64), L, np.array([p[0] for p in props]))
            assert np.all(np.abs(pred - ref_pred) <= 2e-2 * np.maximum(np.abs(ref_pred), 1.0))
            want_rank = sorted(range(24), key=lambda j: (-pred[j], j))[:4]
            assert list(ranked) == want_rank
            best, best_t = None, None
            for r, j in enumerate(ranked):
                Jc, e, v, cu = props[j]
                tt = oracle.tts_eval(L, Jc, betas, R, seed, cu, Sw, 2, 1)[0]
                assert res["tts_new"][r] == tt and res["edge"][r] == e and res["new_value"][r] == v
                if best is None or tt > best_t:
                    best, best_t = r, tt
            keep = best_t > tcur
            assert list(res["accepted"]) == [1 if (keep and r == best) else 0 for r in range(4)]
            if keep:
                Jcur, tcur = props[ranked[best]][0], best_t
            assert h.engineer_tts() == tcur and np.array_equal(h.couplers(), Jcur)


def test_guided_loop_runs_at_c16(P):
    """The guided step at the C_16 shape (48 temperatures in [0.05, 5], 32 runs)."""
    cfg = W.CONFIGS["c16_guided"]
    J = W.random_couplers(16, cfg["seed"], 0)
    betas = W.beta_ladder(cfg["n_temps"], cfg["beta_min"], cfg["beta_max"])
    with P.Surrogate() as m, P.PTHandle(16, J, betas, cfg["n_runs"], cfg["seed"], 0) as h:
        m.set_params(W.surrogate_init_params(1))
        h.engineer_begin(S=256, pass_mult=1, exchange_every=1, base_uid=0)
        res, pred, ranked = h.engineer_guided_step(m, 0, n_prop=cfg["proposals"], top=cfg["top"])
        assert len(set(ranked)) == cfg["top"] and np.all(np.isfinite(pred))
        assert np.all(res["tts_new"] >= 0) and res["accepted"].sum() <= 1
