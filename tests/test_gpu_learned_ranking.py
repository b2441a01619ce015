"""What the trained surrogate adds: ranking of single-coupler moves.

On a fixed C_4 instance (16 temperatures in [0.1, 3], 64 runs, TTS horizon
1024 sweeps with the 4x target pass) every one of the 352 x 5 single-coupler
neighbours is PT-evaluated twice under independent keys.  Of these
measurements, 80 % train the GPU surrogate on differences
(log10 TTS of the neighbour minus that of the instance; guided.train_pairs)
and the rest are held out.  The repeat correlation of the two measurements
bounds what any ranking can reach; the untrained network ranks at chance.

Training is bit-reproducible, but its result still depends on the order in
which the pairs are visited: the held-out rank correlation of single runs
ranges over about 0.15-0.35 across shuffles.  The test therefore trains
three networks (shuffles 0, 1, 2) and asserts on their mean: the trained
networks' rank correlation with the measured held-out differences is at
least 0.25 and at least 0.2 above the untrained network's, it stays below
the repeat correlation of the measurement itself, and picking the
best-predicted 4 of 64 random proposals (first network) finds harder moves
on average than taking 4 at random (the guided step's use of the ranking).
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1605_03607_gb300 as pkg
    from paper_1605_03607_gb300 import build as b
    b.build()
    pkg.load()
    return pkg


def _spearman(a, b):
    ra, rb = np.argsort(np.argsort(a)), np.argsort(np.argsort(b))
    return float(np.corrcoef(ra, rb)[0, 1])


def test_trained_ranking_beats_untrained_on_held_out_moves(P):
    from paper_1605_03607_gb300 import guided as G
    L, NT, R, S, pm, seed = 4, 16, 64, 1024, 4, 777
    betas = W.beta_ladder(NT, 0.1, 3.0)
    J0 = W.random_couplers(L, seed, 10000)
    nb = np.stack([np.where(np.arange(len(J0)) == e, v, J0).astype(np.int8)
                   for e in range(len(J0)) for v in (-3, -2, -1, 1, 2, 3) if v != J0[e]])
    lg = lambda t: np.log10(np.maximum(np.asarray(t, np.float64), 1.0))
    with P.PTHandle(L, J0, betas, R, seed, 0) as h:
        def ev(Js, key0):
            return np.concatenate([h.tts_eval_many(Js[s:s + 256], np.arange(len(Js[s:s + 256])) + key0 + s, S, pm)["tts"]
                                   for s in range(0, len(Js), 256)])
        base = lg(ev(np.repeat(J0[None], 32, 0), 7_000_000)).mean()
        a, b = ev(nb, 1_000_000), ev(nb, 2_000_000)
    assert np.all(a <= S) and np.all(b <= S)
    d = 0.5 * (lg(a) + lg(b)) - base
    repeat = _spearman(a, b)
    perm = np.random.default_rng(0).permutation(len(d))
    tr, va = perm[:1400], perm[1400:]
    with P.Surrogate() as u:
        u.set_params(W.surrogate_init_params(1))
        sp_u = _spearman(u.forward(L, nb[va]), d[va])
    sps, guided, plain = [], [], []
    for shuffle in range(3):
        with P.Surrogate() as m:
            m.set_params(W.surrogate_init_params(1))
            hist = G.train_pairs(m, L, nb[tr], np.repeat(J0[None], len(tr), 0), d[tr] / d[tr].std(), epochs=60,
                                 batch=64, lr=1e-3, seed=shuffle)
            assert hist[-1] < 0.8 * hist[0], hist          # training reduced the pair loss
            sps.append(_spearman(m.forward(L, nb[va]), d[va]))
            if shuffle == 0:                               # the guided step's use of the ranking
                rng = np.random.default_rng(1)
                for _ in range(200):
                    cand = rng.choice(va, 64, replace=False)
                    pc = m.forward(L, nb[cand])
                    guided.append(d[cand[np.argsort(-pc, kind="stable")[:4]]].max())
                    plain.append(d[cand[:4]].max())
    sp_t = float(np.mean(sps))
    assert sp_t >= 0.25 and sp_t >= sp_u + 0.2, (sps, sp_u, repeat)
    assert sp_t < repeat
    assert np.mean(guided) > np.mean(plain), (np.mean(guided), np.mean(plain))
