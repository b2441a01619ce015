"""Pins of the oracle's temperature-random-walk statistics (Sec. III.B).

Each system copy (a configuration, named by the slot it started in) counts the
exchange passes it spends in the hot half (the N_T/2 highest temperatures) and
its completed round trips (back in the coldest slot after reaching the hottest
since its previous visit there).  The pins come from outside the oracle:

* with every coupler 0 every Metropolis flip and every exchange is accepted
  (all energies are 0), so each pass carries the slot-0 copy up the chain to
  the hottest slot and moves every other copy down by one: a rotation whose
  statistics have a closed form;
* every pass puts exactly N_T/2 copies in the hot half;
* a round trip moves a copy N_T - 1 slots up and N_T - 1 down, one slot per
  accepted swap, and an accepted swap moves two copies;
* tracking the walk does not change the trajectory.
"""
import numpy as np
import pytest

import oracle
import workloads as W


def _rotation_stats(NT, M):
    """Closed form for the all-accepting walk after M passes: copy c sits in
    slot (c - m) mod NT after pass m; it is first in slot 0 at pass c0 = c
    (NT for c = 0), reaches the hottest slot at the next pass, and returns to
    slot 0 every NT passes."""
    hot0 = NT - NT // 2
    hot = np.array([sum(1 for m in range(1, M + 1) if (c - m) % NT >= hot0) for c in range(NT)], np.uint64)
    trips = np.zeros(NT, np.uint64)
    for c in range(NT):
        c0 = c if c > 0 else NT
        trips[c] = max(0, (M - c0) // NT) if M >= c0 else 0
    slot_copy = np.array([(t + M) % NT for t in range(NT)], np.int32)
    return hot, trips, slot_copy


@pytest.mark.parametrize("L,NT,R,sweeps,x", [(2, 2, 2, 37, 1), (3, 5, 2, 41, 1), (4, 6, 3, 50, 1),
                                            (2, 16, 2, 200, 1), (2, 7, 2, 120, 10), (1, 4, 3, 33, 3)])
def test_zero_couplers_rotate_copies(L, NT, R, sweeps, x):
    J = np.zeros(W.chimera_n_edges(L), np.int8)
    st = oracle.PTState(L, J, W.beta_ladder(NT, 0.1, 3.0), R, 11, 2, walk=True)
    st.sweeps(sweeps, x)
    M = sweeps // x
    assert st.n_passes == M
    hot, trips, slot_copy = _rotation_stats(NT, M)
    for r in range(R):
        assert np.array_equal(st.hot[r], hot), r
        assert np.array_equal(st.trips[r], trips), r
        assert np.array_equal(st.copy[r], slot_copy), r
    assert np.all(st.E == 0)
    assert np.all(st.xacc[:, :NT - 1] == M)          # every swap accepted


def test_standalone_exchange_rotates_too():
    NT, L = 5, 2
    J = np.zeros(W.chimera_n_edges(L), np.int8)
    st = oracle.PTState(L, J, W.beta_ladder(NT, 0.1, 3.0), 2, 3, 4, walk=True)
    for _ in range(13):
        st.exchange()
    hot, trips, slot_copy = _rotation_stats(NT, 13)
    assert st.n_passes == 13
    assert np.array_equal(st.hot[0], hot) and np.array_equal(st.trips[0], trips)
    assert np.array_equal(st.copy[1], slot_copy)


@pytest.mark.parametrize("L,NT,x", [(4, 16, 1), (4, 9, 1), (3, 12, 10), (2, 30, 1)])
def test_hot_passes_conserved_and_trips_bounded(L, NT, x):
    R, sweeps = 4, 400
    st = oracle.PTState(L, W.random_couplers(L, 5, NT), W.beta_ladder(NT, 0.1, 3.0), R, 5, 1, walk=True)
    st.sweeps(sweeps, x)
    M = sweeps // x
    assert st.n_passes == M
    assert np.all(st.hot.sum(axis=1) == M * (NT // 2))
    assert np.all(st.hot <= M)
    # a round trip is 2 (NT - 1) single-slot moves; an accepted swap is two of them
    assert np.all(st.trips.sum(axis=1) * (NT - 1) <= st.xacc[:, :NT - 1].sum(axis=1))
    # the copy map stays a permutation of the copies
    assert np.all(np.sort(st.copy, axis=1) == np.arange(NT))
    if M >= 200:
        assert st.trips.sum() > 0                     # the ladders do mix over this many passes


def test_tracking_leaves_the_trajectory_unchanged():
    L, NT, R = 4, 12, 3
    J, b = W.random_couplers(L, 9, 0), W.beta_ladder(NT, 0.1, 3.0)
    a = oracle.PTState(L, J, b, R, 9, 0, walk=True)
    c = oracle.PTState(L, J, b, R, 9, 0)
    a.sweeps(60, 2); c.sweeps(60, 2)
    a.exchange(); c.exchange()
    for k in ("spins", "E", "best", "first", "macc", "xacc"):
        assert np.array_equal(getattr(a, k), getattr(c, k)), k


def test_one_temperature_has_no_walk():
    st = oracle.PTState(2, W.random_couplers(2, 1, 0), np.array([1.0]), 2, 1, 0, walk=True)
    st.sweeps(20, 1)
    st.exchange()
    assert st.n_passes == 0 and st.hot.sum() == 0 and st.trips.sum() == 0
