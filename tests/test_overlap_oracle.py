"""Pins of the oracle's ground / first-excited overlap analysis (Sec. III.B):
hand-built replica sets whose samples and overlaps are known by counting."""
import numpy as np

import oracle


def test_identical_complementary_and_one_flip():
    N = 16
    s = np.ones(N, np.int8)
    one_flip = s.copy(); one_flip[3] = -1
    three = s.copy(); three[:3] = -1
    other = -one_flip
    # 4 runs x 2 slots; run 2 and 3 hold the excited states, run 0's warm slot
    # repeats the ground energy (the coldest replica is the sample)
    spins = np.stack([np.stack([s, other]), np.stack([-s, one_flip]), np.stack([one_flip, s]),
                      np.stack([three, s])])
    E = np.array([[-10, -10], [-10, 4], [-8, 4], [-8, 6]])
    r = oracle.overlaps(spins, E, -10)
    # ground samples: run0 slot0 (s), run1 slot0 (-s) -> |q| = 1 (global flip);
    # excited samples (E1 = -8): run2 slot0 (one_flip), run3 slot0 (three)
    assert r["n_gs"] == 2 and r["n_es"] == 2 and r["E1"] == -8
    assert r["q_gs_gs"] == 1.0
    vals = sorted([14 / 16, 14 / 16, 10 / 16, 10 / 16])
    assert r["q_gs_es"] == vals[1]                    # lower median of 4 values


def test_sample_is_the_coldest_replica_at_the_level():
    N = 8
    rng = np.random.default_rng(1)
    spins = rng.choice(np.array([-1, 1], np.int8), size=(3, 3, N))
    E = np.array([[-2, -6, -6], [-4, -4, 0], [0, 2, -4]])
    r = oracle.overlaps(spins, E, -6)
    assert r["n_gs"] == 1 and r["E1"] == -4 and r["n_es"] == 2
    assert r["q_gs_gs"] == -1.0                       # one ground sample: no ground pair
    g = spins[0, 1]                                   # run 0's coldest replica at -6 is slot 1
    h = [int(np.sum(g != spins[1, 0])), int(np.sum(g != spins[2, 2]))]
    assert r["q_gs_es"] == sorted(abs(N - 2 * x) for x in h)[0] / N
    r2 = oracle.overlaps(spins, np.full((3, 3), -6), -6)
    assert r2["n_es"] == 0 and r2["E1"] == 2**31 - 1 and r2["q_gs_es"] == -1.0 and r2["n_gs"] == 3
