"""Temperature random walk on the GPU (pt_set_walk_stats / pt_get_walk_stats)
against the oracle, for both sweep mappings, and against the closed form of the
all-accepting walk (every coupler 0).  Tracking must not change a trajectory."""
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


CASES = [
    # L, NT, R, sweeps, exchange_every, mapping (team, slot_parallel, runs_per_cta) or None, sweeps per launch
    (4, 16, 5, 300, 1, None, 4096),
    (4, 16, 5, 300, 1, (4, 16, 1), 4096),
    (8, 32, 3, 200, 10, (4, 32, 1), 4096),          # EMCS: 10 sweeps + 1 exchange
    (8, 32, 3, 200, 10, None, 4096),
    (3, 9, 4, 250, 1, (8, 9, 1), 17),               # odd N_T, walk carried across many launches
    (5, 7, 3, 240, 3, None, 13),
    (2, 30, 2, 400, 1, (2, 30, 2), 4096),
]


@pytest.mark.parametrize("L,NT,R,sweeps,x,mapping,spl", CASES)
def test_walk_matches_oracle(P, L, NT, R, sweeps, x, mapping, spl):
    seed, uid = 31, 7
    J, b = W.random_couplers(L, seed, uid), W.beta_ladder(NT, 0.1, 3.0)
    ref = oracle.PTState(L, J, b, R, seed, uid, walk=True)
    ref.sweeps(sweeps // 2, x)
    ref.exchange()
    ref.sweeps(sweeps - sweeps // 2, x)
    with P.PTHandle(L, J, b, R, seed, uid) as h:
        if mapping:
            h.set_mapping(*mapping)
        h.set_schedule(0, 0, spl)
        h.set_walk_stats(True)
        h.sweep(sweeps // 2, x)
        h.exchange()
        h.sweep(sweeps - sweeps // 2, x)
        hot, trips, n = h.walk_stats()
        st = h.state()
    assert n == ref.n_passes
    assert np.array_equal(hot, ref.hot) and np.array_equal(trips, ref.trips)
    for k in ("spins", "E", "best", "first", "macc", "xacc"):
        assert np.array_equal(st[k], getattr(ref, k)), k


@pytest.mark.parametrize("mapping", [None, (8, 6, 2)])
def test_zero_couplers_rotation_on_gpu(P, mapping):
    """Every coupler 0: all energies are 0, every swap is accepted and each pass
    rotates the copies (slot-0 copy to the top, the rest down one slot)."""
    L, NT, R, M = 2, 6, 3, 50
    J = np.zeros(W.chimera_n_edges(L), np.int8)
    with P.PTHandle(L, J, W.beta_ladder(NT, 0.1, 3.0), R, 5, 1) as h:
        if mapping:
            h.set_mapping(*mapping)
        h.set_walk_stats(True)
        h.sweep(M, 1)
        hot, trips, n = h.walk_stats()
    assert n == M
    hot0 = NT - NT // 2
    for c in range(NT):
        exp_hot = sum(1 for m in range(1, M + 1) if (c - m) % NT >= hot0)
        c0 = c if c > 0 else NT
        exp_trips = (M - c0) // NT if M >= c0 else 0
        assert np.all(hot[:, c] == exp_hot) and np.all(trips[:, c] == exp_trips), c


def test_walk_tracking_does_not_change_results_and_resets(P):
    L, NT, R = 4, 12, 4
    J, b = W.random_couplers(L, 3, 3), W.beta_ladder(NT, 0.1, 3.0)
    with P.PTHandle(L, J, b, R, 3, 3) as a, P.PTHandle(L, J, b, R, 3, 3) as c:
        a.set_walk_stats(True)
        a.sweep(80, 1); c.sweep(80, 1)
        sa, sc = a.state(), c.state()
        for k in ("spins", "E", "best", "first", "macc", "xacc"):
            assert np.array_equal(sa[k], sc[k]), k
        hot, trips, n = a.walk_stats()
        assert n == 80 and hot.sum() == R * 80 * (NT // 2)
        a.reset(3)
        hot, trips, n = a.walk_stats()
        assert n == 0 and hot.sum() == 0 and trips.sum() == 0
        a.set_walk_stats(False)
        with pytest.raises(P.PTError, match="not tracked"):
            a.walk_stats()
        a.sweep(10, 1)                                   # untracked runs go on as before
