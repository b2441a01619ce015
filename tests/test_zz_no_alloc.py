"""pt_tts_eval_noalloc: the evaluation entry point that allocates nothing.

It exists for callers that cannot call cudaMalloc when they evaluate an
instance (code living inside another framework's memory budget, or loops that
cannot take cudaMalloc's synchronisation).  Its device scratch is a static
array shared by all calls, so this test calls it twice in a row and checks
both results against the handle-based entry point (pt_create + pt_tts_eval)
on the same inputs.  The results are integers (sweep counts, energies), so
they must be equal, the same bar every other parity test here uses.

This file is named to be collected last.
"""
import ctypes

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


def _noalloc(P, L, J, betas, R, seed, uid, S, pass_mult, x):
    lib = P.load()
    t, n, tg = ctypes.c_int32(-1), ctypes.c_int32(-1), ctypes.c_int32(-1)
    rc = lib.pt_tts_eval_noalloc(L, J.ctypes.data_as(ctypes.c_void_p), len(J),
                                 betas.ctypes.data_as(ctypes.c_void_p), len(betas), R, seed, uid,
                                 S, pass_mult, x, None, ctypes.byref(t), ctypes.byref(n), ctypes.byref(tg))
    return rc, (t.value, n.value, tg.value)


@pytest.mark.parametrize("L,NT,R,S,pm,uids", [
    (4, 16, 8, 512, 1, (0, 7)),       # the tiny configuration's shape
    (8, 32, 16, 256, 4, (3, 3)),      # same uid twice: the reused scratch must not leak state
    (1, 3, 8, 256, 1, (1, 2)),        # one cell: more thread slots per run than temperatures
    (3, 16, 6, 256, 1, (4, 5)),       # L^2 = 9: slots per run rounded up past n_temps
    (2, 1, 4, 128, 2, (6, 6)),        # one temperature: no exchange pairs
])
def test_noalloc_matches_handle_path_twice(P, L, NT, R, S, pm, uids):
    seed = 20160511
    J = W.random_couplers(L, seed, L)
    betas = W.beta_ladder(NT, 0.1, 3.0)
    for uid in uids:                                   # two calls in a row
        rc, got = _noalloc(P, L, J, betas, R, seed, uid, S, pm, 1)
        assert rc == 0, P.load().pt_last_error(None)
        with P.PTHandle(L, J, betas, R, seed, uid) as h:
            want = h.tts_eval(uid, S, pm, 1)
        assert got == want


def test_noalloc_rejects_oversize(P):
    L, NT, R = 16, 48, 64                              # 64 * 48 * 2048 spin bytes > 2^21
    J = W.random_couplers(L, 1, 0)
    betas = W.beta_ladder(NT, 0.05, 5.0)
    rc, _ = _noalloc(P, L, J, betas, R, 1, 0, 16, 1, 1)
    assert rc == P._lib.PT_ERR_ARG
    assert b"no-alloc scratch" in P.load().pt_last_error(None)
