"""The bounds-checking debug build (-DPT_DEBUG) on valid inputs.

The debug library checks every data-dependent index its kernels use and
reports a failed check through pt_debug_status instead of faulting.  Here it
runs the main paths on small valid cases -- both sweep mappings, a doubling
TTS evaluation, a speculative RAO batch, a planted instance whose couplers
exceed +-3 (larger Metropolis table), a graph-launched batch and the
allocation-free evaluation -- and must report no failed check and results
equal to the oracle's.  Two long runs with an exchange pass every sweep (48
temperatures on a wide ladder, 64 on a narrow one) also re-derive every
closed-form exchange criterion from the table (code 8 on a difference).  It
runs in a child process because a process loads one build of the library.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys
sys.path.insert(0, ROOT)
import numpy as np
from paper_1605_03607_gb300 import build as b
b.build(debug=True)
import paper_1605_03607_gb300 as P
import oracle
import workloads as W
assert P.debug_enabled(), "not the debug build"
L, NT, R, seed = 4, 8, 4, 20160519
betas = W.beta_ladder(NT, 0.1, 3.0)
J = W.random_couplers(L, seed, 0)
for mapping in (None, (4, 8, 2)):
    with P.PTHandle(L, J, betas, R, seed, 1) as h:
        if mapping:
            h.set_mapping(*mapping)
        h.sweep(90, 1)
        h.exchange()
        st = h.state()
    ref = oracle.PTState(L, J, betas, R, seed, 1)
    ref.sweeps(90, 1)
    ref.exchange()
    assert np.array_equal(st["spins"], ref.spins) and np.array_equal(st["E"], ref.E)
    assert np.array_equal(st["best"], ref.best) and np.array_equal(st["first"], ref.first)
with P.PTHandle(L, J, betas, R, seed, 2) as h:
    assert h.tts_eval_doubling(3, 16, 256) == oracle.tts_eval_doubling(L, J, betas, R, seed, 3, 16, 256)
    h.engineer_begin(S=32, pass_mult=2)
    h.engineer_run(0, 6, 3)
    h.lao_begin(64, 5, 60, 5)
    h.lao_run(1, 4, 2)
    assert h.table_rows() > 19
insts = [dict(L=l, J=W.random_couplers(l, seed, i), betas=W.beta_ladder(nt, 0.1, 3.0), uid=i)
         for i, (l, nt) in enumerate([(2, 6), (4, 8), (4, 12), (8, 16)])]
with P.PTBatch(insts, 4, seed) as bt:
    bt.reset()
    bt.run(64, 1)
    s0 = bt.state(1)
ref = oracle.PTState(4, insts[1]["J"], insts[1]["betas"], 4, seed, 1)
ref.sweeps(64, 1)
assert np.array_equal(s0["spins"], ref.spins) and np.array_equal(s0["E"], ref.E)
import ctypes
lib = P.load()
t = ctypes.c_int32()
assert lib.pt_tts_eval_noalloc(L, J.ctypes.data_as(ctypes.c_void_p), len(J), betas.ctypes.data_as(ctypes.c_void_p),
                               NT, R, seed, 7, 64, 1, 1, None, ctypes.byref(t), None, None) == 0
assert t.value == oracle.tts_eval(L, J, betas, R, seed, 7, 64, 1, 1)[0]
# exchange every sweep over many criteria: the debug build recomputes each
# closed-form critical gap by the table search (code 8 on any difference)
for (l, nt, lo, hi, runs, n) in ((4, 48, 0.05, 5.0, 64, 1500), (2, 64, 0.30, 0.35, 64, 1500)):
    with P.PTHandle(l, W.random_couplers(l, seed, 9), W.beta_ladder(nt, lo, hi), runs, seed, 9) as h:
        h.sweep(n, 1)
        assert P.debug_status() == 0, "closed-form exchange criterion differs from the table search"
code = P.debug_status()
assert code == 0, f"bounds check {code} failed"
print("debug build: no failed bounds check")
'''


def test_debug_build_runs_clean_on_valid_inputs():
    env = dict(os.environ, PT_GB300_DEBUG="1")
    r = subprocess.run([sys.executable, "-c", f"ROOT = {ROOT!r}\n" + SCRIPT], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-3000:]
    assert "no failed bounds check" in r.stdout
    assert "PT_DEBUG" not in r.stderr
