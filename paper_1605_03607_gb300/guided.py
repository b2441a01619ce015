"""Surrogate-guided instance engineering: data, training and the two loops.

Orchestration only (every PT sweep, TTS reduction, surrogate forward/backward
and Adam update runs in the library's kernels):

* train: minibatch Adam on (couplers, log10 TTS) pairs with the GPU surrogate.
* train_pairs: minibatch Adam on differences between a candidate and the
  instance it was drawn from -- the form in which the loop's own evaluations
  teach the network which single-coupler moves make an instance harder.
* run_loop: one engineering loop for a number of GPU-seconds, plain,
  ranked by a fixed network, or ranked by a network retrained online on the
  loop's own evaluations; PT decides every kept move under the same rule.
"""
from __future__ import annotations

import time

import numpy as np


def log10_tts(tts):
    return np.log10(np.maximum(np.asarray(tts, np.float64), 1.0))


def train(model, L, J, y, epochs=20, batch=256, lr=1e-3, seed=0, standardize=True):
    """Minibatch Adam on (J, y); returns the mean training loss of every epoch.

    standardize: the network is fitted to (y - mean) / std of the training
    targets (the loss history is in those units), so the readout does not
    spend its first thousand steps moving its bias to the targets' level.
    Predictions are then in standardized units, which keeps every ranking;
    `target_scale(y)` gives the (mean, std) to map them back."""
    rng = np.random.default_rng(seed)
    n = len(y)
    y = np.asarray(y, np.float64)
    if standardize:
        mu, sd = target_scale(y)
        y = (y - mu) / sd
    hist = []
    for _ in range(epochs):
        perm = rng.permutation(n)
        losses = []
        for s in range(0, n, batch):
            idx = perm[s:s + batch]
            losses.append(model.train_step(L, J[idx], y[idx].astype(np.float32), lr))
        hist.append(float(np.mean(losses)))
    return hist


def train_pairs(model, L, J_cand, J_base, d, epochs=60, batch=64, lr=1e-3, seed=0):
    """Minibatch Adam on differences: the network f is fitted so that
    f(J_cand[i]) - f(J_base[i]) matches d[i] (a candidate's log10 TTS minus
    that of the instance it was drawn from, in whatever units d is given).

    A single-coupler move changes the pooled representation of a graph by a
    fraction of a percent, so an absolute-target fit is dominated by the
    part every graph shares; the pairwise loss sum_i (f(J'_i) - f(J_i) - d_i)^2
    removes that part.  Each step runs the library's forward on the batch of
    candidates and their bases, then one train_step whose per-graph targets
    are chosen so that its mean-squared-error gradient equals the gradient of
    the pairwise loss: for a candidate, (y - t) = r (n / b), for its base
    (y - t) = -r (n / b), with r the pair's residual, b pairs and n = 2b
    graphs in the batch.  Returns the mean squared residual of every epoch."""
    rng = np.random.default_rng(seed)
    J_cand = np.asarray(J_cand, np.int8)
    J_base = np.asarray(J_base, np.int8)
    d = np.asarray(d, np.float64)
    n = len(d)
    hist = []
    for _ in range(epochs):
        perm = rng.permutation(n)
        losses = []
        for s in range(0, n, batch):
            idx = perm[s:s + batch]
            b = len(idx)
            graphs = np.concatenate([J_cand[idx], J_base[idx]])
            y = model.forward(L, graphs).astype(np.float64)
            r = (y[:b] - y[b:]) - d[idx]
            t = np.concatenate([y[:b] - r * 2.0, y[b:] + r * 2.0])
            model.train_step(L, graphs, t.astype(np.float32), lr)
            losses.append(float(np.mean(r * r)))
        hist.append(float(np.mean(losses)))
    return hist


def target_scale(y):
    """(mean, std) used by train(standardize=True)."""
    y = np.asarray(y, np.float64)
    return float(y.mean()), float(max(y.std(), 1e-6))


def run_loop(h, L, seconds, model=None, online=False, step0=0, n_prop=64, top=4, retrain_every=8,
             min_pairs=32, epochs=4, lr=1e-3, window=1024, max_steps=10**9):
    """One engineering loop for `seconds` of GPU time (host wall clock around
    the synchronous library calls, training included).  Every step draws
    n_prop proposals, PT-evaluates `top` of them in one batched launch and
    keeps the one with the largest TTS if it beats the current TTS
    (engineer_guided_step): the same acceptance rule in every arm.

    model None: the plain loop (proposals 0..top-1, no ranking).  model given:
    its ranking picks the `top`; with online=True it is retrained every
    `retrain_every` steps (train_pairs, `epochs` passes) on the `window` most
    recent pairs the loop has evaluated: (candidate, instance it was drawn
    from, log10 TTS difference), and until its first training it does not
    rank (the plain choice), so an untrained network's bias never steers the
    loop.  Returns (trace [(seconds, tts, steps)], pairs evaluated)."""
    trace = [(0.0, h.engineer_tts(), 0)]
    Jc, Jb, d = [], [], []
    used, step = 0.0, step0
    trained = False
    while used < seconds and step - step0 < max_steps:
        J = h.couplers()
        tcur = h.engineer_tts()
        t0 = time.perf_counter()
        ranker = model if (model is not None and (trained or not online)) else None
        res, _, _ = h.engineer_guided_step(ranker, step, n_prop, top)
        for r in range(top):
            c = J.copy()
            c[res["edge"][r]] = res["new_value"][r]
            Jc.append(c)
            Jb.append(J)
            d.append(float(log10_tts(res["tts_new"][r]) - log10_tts(tcur)))
        step += 1
        if online and model is not None and (step - step0) % retrain_every == 0 and len(d) >= min_pairs:
            dd = np.asarray(d[-window:])
            train_pairs(model, L, np.asarray(Jc[-window:]), np.asarray(Jb[-window:]), dd / max(dd.std(), 1e-6),
                        epochs=epochs, batch=64, lr=lr, seed=step)
            trained = True
        used += time.perf_counter() - t0
        trace.append((used, h.engineer_tts(), step - step0))
    return trace, len(d)


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
