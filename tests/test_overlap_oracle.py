"""Pins of the oracle's ground / first-excited overlap analysis (Sec. III.B):
hand-built samples whose overlaps are known by counting."""
import numpy as np

import oracle


def test_identical_complementary_and_one_flip():
    N = 16
    s = np.ones(N, np.int8)
    one_flip = s.copy(); one_flip[3] = -1
    three = s.copy(); three[:3] = -1
    samples = np.stack([s, -s, one_flip, three])
    E = np.array([-10, -10, -8, -8])
    r = oracle.overlaps(samples, E, -10)
    # ground pair (s, -s): h = N -> |q| = 1 (global flip); (ground, excited) pairs:
    # s/one_flip 1 - 2/16, -s/one_flip |1 - 30/16|, s/three 1 - 6/16, -s/three |1 - 26/16|
    assert r["n_gs"] == 2 and r["n_es"] == 2 and r["E1"] == -8
    assert r["q_gs_gs"] == 1.0
    vals = sorted([14 / 16, 14 / 16, 10 / 16, 10 / 16])
    assert r["q_gs_es"] == vals[1]                    # lower median of 4 values


def test_lowest_level_above_ground_and_missing_pairs():
    N = 8
    rng = np.random.default_rng(1)
    samples = rng.choice(np.array([-1, 1], np.int8), size=(5, N))
    E = np.array([-6, -2, -4, -4, 0])
    r = oracle.overlaps(samples, E, -6)
    assert r["n_gs"] == 1 and r["E1"] == -4 and r["n_es"] == 2
    assert r["q_gs_gs"] == -1.0                       # one ground sample: no ground pair
    h = [int(np.sum(samples[0] != samples[k])) for k in (2, 3)]
    assert r["q_gs_es"] == sorted(abs(N - 2 * x) for x in h)[0] / N
    r2 = oracle.overlaps(samples, np.full(5, -6), -6)
    assert r2["n_es"] == 0 and r2["E1"] == 2**31 - 1 and r2["q_gs_es"] == -1.0
