"""Surrogate-guided instance engineering: data, training and the two loops.

Orchestration only (every PT sweep, TTS reduction, surrogate forward/backward
and Adam update runs in the library's kernels):

* collect_pairs: runs the plain RAO loop (Algorithm 1, speculative batches)
  on seed instances and keeps every PT-evaluated candidate as a training pair
  (couplers, log10 TTS) -- the loop produces its own training data.
* train: minibatch Adam on those pairs with the GPU surrogate.
* run_plain / run_guided: the two loops on the same seed instance for a given
  number of GPU-seconds (wall clock around the synchronous library calls);
  PT decides every kept move in both.
"""
from __future__ import annotations

import time

import numpy as np

from ._lib import PTHandle


def log10_tts(tts):
    return np.log10(np.maximum(np.asarray(tts, np.float64), 1.0))


def _one_loop(L, J0, betas, n_runs, seed, uid, S, pass_mult, steps, speculation):
    Js, ys = [], []
    with PTHandle(L, J0, betas, n_runs, seed, uid) as h:
        t0 = h.engineer_begin(S=S, pass_mult=pass_mult, exchange_every=1, base_uid=uid)
        J = np.asarray(J0, np.int8).copy()
        Js.append(J.copy())
        ys.append(t0)
        res = h.engineer_run(0, steps, speculation)
        for k in range(steps):
            Jc = J.copy()
            Jc[res["edge"][k]] = res["new_value"][k]
            Js.append(Jc)
            ys.append(int(res["tts_new"][k]))
            if res["accepted"][k]:
                J = Jc
    return Js, ys


def collect_pairs(L, J0s, betas, n_runs, seed, uids, S, pass_mult, steps, speculation=16, workers=4):
    """Plain RAO from each seed instance; returns (J [n, E] int8, y [n] log10 TTS, tts [n]).

    `workers` loops run at once from host threads, each on its own handle and
    stream (the library calls release the interpreter), to keep the GPU full."""
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=max(1, workers)) as ex:
        parts = list(ex.map(lambda a: _one_loop(L, a[0], betas, n_runs, seed, a[1], S, pass_mult, steps,
                                                speculation), zip(J0s, uids)))
    Js = [j for p in parts for j in p[0]]
    ys = [y for p in parts for y in p[1]]
    tts = np.array(ys, np.int64)
    return np.array(Js, np.int8), log10_tts(tts), tts


def train(model, L, J, y, epochs=20, batch=256, lr=1e-3, seed=0, standardize=True):
    """Minibatch Adam on (J, y); returns the mean training loss of every epoch."""
    rng = np.random.default_rng(seed)
    n = len(y)
    hist = []
    for _ in range(epochs):
        perm = rng.permutation(n)
        losses = []
        for s in range(0, n, batch):
            idx = perm[s:s + batch]
            losses.append(model.train_step(L, J[idx], y[idx].astype(np.float32), lr))
        hist.append(float(np.mean(losses)))
    return hist


def run_plain(h, seconds, step0=0, speculation=16, max_steps=10**9):
    """Plain RAO for `seconds` of GPU time; returns a trace of (seconds, tts, steps)."""
    trace = [(0.0, h.engineer_tts(), 0)]
    used, step = 0.0, step0
    while used < seconds and step - step0 < max_steps:
        t0 = time.perf_counter()
        h.engineer_run(step, speculation, speculation)
        used += time.perf_counter() - t0
        step += speculation
        trace.append((used, h.engineer_tts(), step - step0))
    return trace


def run_guided(h, model, seconds, step0=0, n_prop=64, top=4, max_steps=10**9, pairs=None):
    """Surrogate-guided RAO for `seconds` of GPU time; evaluated candidates are
    appended to `pairs` (list of (J, tts)) when given."""
    trace = [(0.0, h.engineer_tts(), 0)]
    used, step = 0.0, step0
    while used < seconds and step - step0 < max_steps:
        J = h.couplers()
        t0 = time.perf_counter()
        res, pred, ranked = h.engineer_guided_step(model, step, n_prop, top)
        used += time.perf_counter() - t0
        if pairs is not None:
            for r in range(top):
                Jc = J.copy()
                Jc[res["edge"][r]] = res["new_value"][r]
                pairs.append((Jc, int(res["tts_new"][r])))
        step += 1
        trace.append((used, h.engineer_tts(), step - step0))
    return trace


def gain_per_second(trace, cap=None):
    """(log10 TTS - log10 TTS_initial) / GPU-seconds, up to the first point where
    the TTS reaches `cap` (the unsolved value S + 1, beyond which no move can
    count as harder) or to the end of the trace."""
    end = len(trace) - 1
    if cap is not None:
        for i, (_, tts, _) in enumerate(trace):
            if tts >= cap:
                end = i
                break
    t_end, tts_end, _ = trace[end]
    return (log10_tts(tts_end) - log10_tts(trace[0][1])) / max(t_end, 1e-9)
