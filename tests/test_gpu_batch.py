"""Batched PT (persistent, graph-captured launch) vs the CPU oracle.

Each instance of a batch keeps its own key (seed, uid), so its runs must be
bit-identical to the oracle (and to a single-instance handle) whatever the
batch composition, schedule, or split of the sweeps into runs.
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


MIXED = [(4, 5), (8, 6), (12, 4), (5, 3), (16, 3), (3, 7), (1, 4), (4, 16), (2, 2), (6, 1)]


def _mixed(seed=91):
    out = []
    for i, (L, nt) in enumerate(MIXED):
        out.append(dict(L=L, J=W.random_couplers(L, seed, i), betas=W.beta_ladder(nt, 0.1, 3.0),
                        uid=1000 + i))
    return out


def _check_instance(bst, x, R, seed, sweeps, ctx):
    ref = oracle.PTState(x["L"], x["J"], x["betas"], R, seed, x["uid"])
    ref.sweeps(sweeps, 1)
    for k in ("spins", "E", "best", "first", "macc"):
        assert np.array_equal(bst[k], getattr(ref, k)), f"{ctx}: {k}"
    if len(x["betas"]) > 1:
        assert np.array_equal(bst["xacc"], ref.xacc), f"{ctx}: xacc"
    return ref


def test_mixed_batch_bit_exact(P):
    seed, R = 91, 3
    inst = _mixed(seed)
    with P.PTBatch(inst, R, seed) as b:
        b.run(25, 1)
        b.run(15, 1)                                   # graph replay with a patched sweep counter
        t, h, tg = b.tts(40)
        for i, x in enumerate(inst):
            ref = _check_instance(b.state(i), x, R, seed, 40, f"instance {i} L={x['L']}")
            assert (t[i], h[i], tg[i]) == oracle.tts(ref.best, ref.first, oracle.TARGET_BEST, 40)


def test_batch_equals_single_handle(P):
    seed, R = 92, 4
    inst = _mixed(seed)[:3]
    with P.PTBatch(inst, R, seed) as b:
        b.run(30, 1)
        for i, x in enumerate(inst):
            with P.PTHandle(x["L"], x["J"], x["betas"], R, seed, x["uid"]) as h:
                h.sweep(30, 1)
                a, s = b.state(i), h.state()
                for k in ("spins", "E", "best", "first", "macc", "xacc"):
                    assert np.array_equal(a[k], s[k]), k


def test_batch_schedule_and_autotune_invariance(P):
    seed, R = 93, 4
    inst = _mixed(seed)
    states = []
    with P.PTBatch(inst, R, seed) as b:
        b.run(24, 1)
        states.append([b.state(i) for i in range(len(inst))])
        for block, L, sp, ipc in ((256, 4, 2, 4), (512, 8, 1, 2), (1024, 16, 1, 1), (512, 12, 2, 1)):
            b.set_schedule(block, L, sp, ipc)
            b.reset()
            b.run(24, 1)
            states.append([b.state(i) for i in range(len(inst))])
        b.autotune(trial_sweeps=4)
        b.run(24, 1)
        states.append([b.state(i) for i in range(len(inst))])
    for st in states[1:]:
        for i in range(len(inst)):
            for k in ("spins", "E", "best", "first", "macc", "xacc"):
                assert np.array_equal(st[i][k], states[0][i][k]), (i, k)


def test_slot_major_batch_bit_exact(P):
    """The whole batch on the slot-major mapping (one kernel instantiation per
    launch), default schedules and several per-size team layouts, against the
    oracle and against the cell-major batch."""
    seed, R = 94, 3
    inst = _mixed(seed)
    with P.PTBatch(inst, R, seed) as b:
        b.run(30, 1)
        cell = [b.state(i) for i in range(len(inst))]
        b.set_mapping(4)                                 # switch only: defaults for every size
        assert all(b.mapping(x["L"]) > 0 for x in inst)
        b.reset()
        b.run(18, 1)
        b.run(12, 1)
        for i, x in enumerate(inst):
            _check_instance(b.state(i), x, R, seed, 30, f"slot-major instance {i} L={x['L']}")
        layouts = ((4, 2, 16, 2), (8, 8, 4, 1), (16, 16, 2, 1), (12, 32, 2, 2), (1, 8, 4, 1),
                   (4, 32, 1, 3))
        for L, team, sp, ipc in layouts:
            b.set_mapping(team, L, sp, ipc)
            assert b.mapping(L) == team and b.schedule(L)[1:] == (sp, min(ipc, R))
            b.reset()
            b.run(30, 1)
            for i in range(len(inst)):
                st = b.state(i)
                for k in ("spins", "E", "best", "first", "macc", "xacc"):
                    assert np.array_equal(st[k], cell[i][k]), (L, team, sp, ipc, i, k)
        b.set_mapping(0)                                 # back to cell-major
        assert b.mapping(4) == 0
        b.reset()
        b.run(30, 1)
        for i in range(len(inst)):
            assert np.array_equal(b.state(i)["spins"], cell[i]["spins"]), i


def test_slot_major_uneven_temperatures(P):
    """One size whose instances have 8..32 temperatures: on the slot-major
    mapping each instance gets teams in proportion to its slots and more runs
    per CTA where that frees threads; every instance matches the oracle."""
    seed, R = 95, 5
    inst = [dict(L=4, J=W.random_couplers(4, seed, i), betas=W.beta_ladder(nt, 0.1, 3.0), uid=2000 + i)
            for i, nt in enumerate((8, 13, 32, 20))]
    with P.PTBatch(inst, R, seed) as b:
        for team, sp, ipc in ((8, 16, 1), (4, 16, 2), (2, 32, 1)):
            b.set_mapping(team, 4, sp, ipc)
            b.reset()
            b.run(40, 1)
            for i, x in enumerate(inst):
                _check_instance(b.state(i), x, R, seed, 40, f"team {team} sp {sp} ipc {ipc} instance {i}")


def test_batch_mapping_rejects_misfits(P):
    inst = _mixed(5)[:3]                                 # sizes 4, 8, 12
    with P.PTBatch(inst, 2, 5) as b:
        with pytest.raises(P.PTError, match="power of two"):
            b.set_mapping(6, 4, 8, 1)
        with pytest.raises(P.PTError, match="fit"):
            b.set_mapping(4, 8, 4, 1)                    # 16 threads per run
        with pytest.raises(P.PTError, match="fit"):
            b.set_schedule(0, 12, 4, 2)                  # cell-major: 2 runs x 576 threads > 1024
        b.set_mapping(4, 8, 8, 1)
        with pytest.raises(P.PTError, match="fit"):
            b.set_schedule(1024, 8, 8, 1)                # slot-major CTAs hold <= 768 threads
        assert b.mapping(8) == 4 and b.schedule(8)[1:] == (8, 1)   # failures change nothing
        with pytest.raises(P.PTError, match="no instance"):
            b.set_mapping(4, 7, 8, 1)


def test_batched_config_shape_sampled(P):
    """The batched configuration (256 instances, C_4/8/12/16, 24..48 temperatures,
    32 runs): a short run compared with the oracle on one instance of each size,
    and energies of sampled replicas of every instance recomputed."""
    cfg = W.CONFIGS["batched_256"]
    inst = W.batched_instances(cfg)
    with P.PTBatch(inst, cfg["n_runs"], cfg["seed"]) as b:
        b.autotune(trial_sweeps=2)
        b.run(12, 1)
        info = b.info()
        assert info["bundles"] > 0 and info["grid"] > 0
        for i in (1, 64, 128, 255):
            x = inst[i]
            _check_instance(b.state(i), x, cfg["n_runs"], cfg["seed"], 12, f"instance {i}")
        for i in range(0, 256, 17):
            st = b.state(i)
            x = inst[i]
            for r, t in ((0, 0), (31, len(x["betas"]) - 1)):
                assert st["E"][r, t] == oracle.energy(x["L"], x["J"], st["spins"][r, t])


def test_batch_rejects_bad_instances(P):
    inst = _mixed(1)[:2]
    inst[1] = dict(inst[1], betas=np.array([1.0, 2.0]))
    with pytest.raises(P.PTError, match="descending"):
        P.PTBatch(inst, 2, 1)
