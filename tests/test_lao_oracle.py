"""Pins of the planted-solution instances and loop adaptive optimisation
(Sec. IV, Algorithm 2), and the library's host-side planting against the oracle.

The pins come from outside the oracle's LAO code: exact ground-state energies by
enumeration (C_1, C_2), the graph itself (every loop is a simple cycle of Chimera
edges), the frustration of each loop, the coupler sum, and the draw
frequencies the construction states (length 4 with probability 0.1).
"""
import numpy as np
import pytest

import oracle
import workloads as W


def _graph(L):
    ei, ej = oracle.chimera_edges(L)
    return ei, ej, {frozenset((int(a), int(b))): e for e, (a, b) in enumerate(zip(ei, ej))}


def _check_loops(L, planted, loops, J, w_max):
    ei, ej, emap = _graph(L)
    Jsum = np.zeros(len(ei), np.int64)
    for rec in loops:
        n, w, f = int(rec[0]), int(rec[1]), int(rec[2])
        assert n in (4, 6) and 1 <= w <= w_max and 0 <= f < n
        edges = [int(e) for e in rec[3:3 + n]]
        assert all(e >= 0 for e in edges) and all(int(e) == -1 for e in rec[3 + n:])
        # a simple cycle: every vertex has degree 2 in the loop, and the edges are connected
        deg = {}
        for e in edges:
            for v in (int(ei[e]), int(ej[e])):
                deg[v] = deg.get(v, 0) + 1
        assert len(edges) == len(set(edges)) and len(deg) == n and all(d == 2 for d in deg.values())
        # exactly the frustrated position violates the planted state
        for m, e in enumerate(edges):
            term = (1 if m == f else -1) * w * planted[ei[e]] * planted[ej[e]]
            Jsum[e] += term
            assert (term * planted[ei[e]] * planted[ej[e]] > 0) == (m == f)
    assert np.array_equal(Jsum, J.astype(np.int64))
    # the engine's bounds: int8 couplers, every spin's sum of |J| <= 127
    assert np.abs(J.astype(np.int64)).max() <= 127
    spin_sum = np.zeros(8 * L * L, np.int64)
    np.add.at(spin_sum, ei, np.abs(J.astype(np.int64)))
    np.add.at(spin_sum, ej, np.abs(J.astype(np.int64)))
    assert spin_sum.max() <= 127 and spin_sum.max() == oracle.coupler_kmax(L, J)
    return spin_sum.max()


@pytest.mark.parametrize("L,M,w", [(1, 2, 5), (1, 3, 5), (2, 8, 5), (2, 12, 5), (2, 12, 3)])
def test_planted_state_is_a_ground_state(L, M, w):
    for uid in range(5):
        planted, loops, J, eg = oracle.lao_plant(L, 20160516, uid, M, w)
        assert eg == -sum(int(w_) * (int(n) - 2) for n, w_ in loops[:, :2])
        assert oracle.energy(L, J, planted) == eg
        assert oracle.ground_energy_bipartite(L, J) == eg          # exact, by enumeration
        _check_loops(L, planted, loops, J, w)


def test_loop_statistics_c8():
    """The paper's parameters (Sec. IV, Fig. 7): 350 loops on C_8, integer
    weights uniform in [1, 5]."""
    lengths, weights, sums = [], [], []
    for uid in range(4):
        planted, loops, J, eg = oracle.lao_plant(8, 20160516, uid, 350, 5)
        sums.append(_check_loops(8, planted, loops, J, 5))
        assert oracle.energy(8, J, planted) == eg
        lengths += list(loops[:, 0]); weights += list(loops[:, 1])
    f4 = np.mean(np.array(lengths) == 4)
    assert abs(f4 - 0.1) < 0.035                                    # 1400 loops: sd 0.008
    counts = np.bincount(weights, minlength=6)[1:]
    assert set(weights) == {1, 2, 3, 4, 5} and counts.min() > 0.15 * 1400
    # the engine's bound on a spin's sum of |J| (127) is far from reached
    assert max(sums) < 100


def test_lao_steps_keep_the_planted_ground_state():
    L, M = 2, 10
    st = oracle.LAOState(L, W.beta_ladder(6, 0.1, 3.0), 4, 20160516, 3, M, S=128, beta_rao=0.5)
    res = st.run(1, 12)
    assert res["accepted"].sum() >= 1
    _check_loops(L, st.planted, st.loops, st.J, 5)
    assert st.E_gs == -sum(int(w) * (int(n) - 2) for n, w in st.loops[:, :2])
    assert oracle.energy(L, st.J, st.planted) == st.E_gs == oracle.ground_energy_bipartite(L, st.J)
    # the logged candidate energies are the formula of each candidate's loops
    assert np.all(res["E_gs"] <= 0)


@pytest.mark.parametrize("L,M,w", [(1, 3, 3), (2, 12, 2), (4, 60, 3), (4, 60, 5), (8, 350, 5)])
def test_library_planting_equals_oracle(L, M, w):
    """Host logic of the library (no GPU work) against the oracle."""
    P = pytest.importorskip("paper_1605_03607_gb300")
    try:
        P.load()
    except RuntimeError:
        pytest.skip("library not built")
    a = P.lao_plant(L, 20160516, 9, M, w)
    b = oracle.lao_plant(L, 20160516, 9, M, w)
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y)
    assert a[3] == b[3]
