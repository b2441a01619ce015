"""CPU oracle (TEST INFRASTRUCTURE ONLY).

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline leg may
import this package.  It is a ctypes binding to ``pt_oracle.c`` (plain C, one
thread, written from the paper) plus the FP64 surrogate oracle in
``surrogate.py``.  It never imports the CUDA package and the CUDA package never
imports it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pt_oracle.c")
_LIB = os.path.join(_HERE, "libpt_oracle.so")

TARGET_BEST = 2**31 - 1
KMAX = 18


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no architecture flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _declare(_lib)
    return _lib


def _p(dtype):
    return np.ctypeslib.ndpointer(dtype=dtype, flags="C_CONTIGUOUS")


def _declare(L):
    c = ctypes
    L.or_philox4x32_10.argtypes = [_p(np.uint32), _p(np.uint32), _p(np.uint32)]
    L.or_chimera_n_edges.argtypes = [c.c_int]
    L.or_chimera_edges.argtypes = [c.c_int, _p(np.int32), _p(np.int32)]
    L.or_spin_colour.argtypes = [c.c_int, c.c_int]
    L.or_energy.argtypes = [c.c_int, _p(np.int8), _p(np.int8)]
    L.or_energy.restype = c.c_int32
    L.or_metropolis_thresholds.argtypes = [c.c_int, _p(np.float64), c.c_int, _p(np.uint32)]
    L.or_coupler_kmax.argtypes = [c.c_int, _p(np.int8)]
    L.or_exchange_thresholds.argtypes = [c.c_int, _p(np.float64), c.c_void_p, c.c_void_p]
    L.or_exchange_thresholds.restype = c.c_int64
    L.or_pt_init_spins.argtypes = [c.c_int, c.c_int, c.c_int, c.c_uint32, c.c_uint32, _p(np.int8)]
    L.or_pt_start.argtypes = [c.c_int, _p(np.int8), c.c_int, c.c_int, _p(np.int8),
                              _p(np.int32), _p(np.int32), _p(np.int32)]
    L.or_pt_sweeps.argtypes = [c.c_int, _p(np.int8), c.c_int, _p(np.float64), c.c_int,
                               c.c_uint32, c.c_uint32, _p(np.int8), _p(np.int32), _p(np.int32),
                               _p(np.int32), _p(np.uint64), _p(np.uint64), c.c_uint32,
                               c.c_int, c.c_int]
    L.or_pt_exchange.argtypes = [c.c_int, _p(np.int8), c.c_int, _p(np.float64), c.c_int,
                                 c.c_uint32, c.c_uint32, _p(np.int8), _p(np.int32),
                                 _p(np.uint64), c.c_uint32]
    L.or_pt_sweeps_walk.argtypes = L.or_pt_sweeps.argtypes + [_p(np.int32), _p(np.uint64), _p(np.uint64),
                                                             _p(np.uint8)]
    L.or_pt_exchange_walk.argtypes = L.or_pt_exchange.argtypes + [_p(np.int32), _p(np.uint64), _p(np.uint64),
                                                                 _p(np.uint8)]
    L.or_lao_plant.argtypes = [c.c_int, c.c_uint32, c.c_uint32, c.c_int, c.c_int, _p(np.int8), _p(np.int32),
                               _p(np.int8), c.POINTER(c.c_int32)]
    L.or_lao_run.argtypes = [c.c_int, c.c_int, _p(np.float64), c.c_int, c.c_uint32, c.c_uint32, c.c_int, c.c_int,
                             c.c_int32, c.c_int, c.c_double, c.c_int, c.c_uint32, c.c_int, _p(np.int8),
                             _p(np.int32), _p(np.int8), c.POINTER(c.c_int32), c.POINTER(c.c_int32),
                             _p(np.int32), _p(np.int32), _p(np.int32), _p(np.int32)]
    L.or_tts.argtypes = [c.c_int, _p(np.int32), _p(np.int32), c.c_int32, c.c_int32,
                         c.POINTER(c.c_int32), c.POINTER(c.c_int32), c.POINTER(c.c_int32)]
    L.or_tts_eval.argtypes = [c.c_int, _p(np.int8), c.c_int, _p(np.float64), c.c_int,
                              c.c_uint32, c.c_uint32, c.c_int32, c.c_int32, c.c_int,
                              c.POINTER(c.c_int32), c.POINTER(c.c_int32), c.POINTER(c.c_int32)]
    L.or_engineer_draw.argtypes = [c.c_int, _p(np.int8), c.c_uint32, c.c_uint32, c.c_uint32,
                                   c.c_uint32, c.POINTER(c.c_int32), c.POINTER(c.c_int32),
                                   c.POINTER(c.c_uint32), c.POINTER(c.c_uint32)]
    L.or_engineer_run.argtypes = [c.c_int, _p(np.int8), c.c_int, _p(np.float64), c.c_int,
                                  c.c_uint32, c.c_uint32, c.c_int32, c.c_int32, c.c_int,
                                  c.c_uint32, c.c_int, c.c_double, c.c_int,
                                  c.POINTER(c.c_int32)] + [c.c_void_p] * 5
    L.or_engineer_run_budget.argtypes = [c.c_int, _p(np.int8), c.c_int, _p(np.float64), c.c_int,
                                         c.c_uint32, c.c_uint32, c.c_int32, c.c_int32, c.c_int32, c.c_int,
                                         c.c_uint32, c.c_int, c.c_double, c.c_int,
                                         c.POINTER(c.c_int32)] + [c.c_void_p] * 5
    L.or_engineer_run_adaptive.argtypes = [c.c_int, _p(np.int8), c.c_int, _p(np.float64), c.c_uint32, c.c_uint32,
                                           c.c_int32, c.c_int32, c.c_int32, c.c_int, c.c_uint32, c.c_int,
                                           c.c_double, c.c_double, c.c_int, c.c_int32, c.c_int64,
                                           c.POINTER(c.c_int32), c.POINTER(c.c_int32)] + [c.c_void_p] * 6
    L.or_tts_eval_doubling.argtypes = [c.c_int, _p(np.int8), c.c_int, _p(np.float64), c.c_int,
                                       c.c_uint32, c.c_uint32, c.c_int32, c.c_int32, c.c_int,
                                       c.POINTER(c.c_int32), c.POINTER(c.c_int32), c.POINTER(c.c_int32),
                                       c.POINTER(c.c_int32)]
    L.or_rao_accept.argtypes = [c.c_int32, c.c_int32, c.c_int, c.c_double, c.c_uint32]
    L.or_ground_energy_bipartite.argtypes = [c.c_int, _p(np.int8)]
    L.or_ground_energy_bipartite.restype = c.c_int32


def _u32(x):
    return int(x) & 0xFFFFFFFF


def philox4x32_10(ctr, key):
    out = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def chimera_edges(L):
    E = lib().or_chimera_n_edges(L)
    ei = np.zeros(E, np.int32)
    ej = np.zeros(E, np.int32)
    lib().or_chimera_edges(L, ei, ej)
    return ei, ej


def spin_colours(L):
    return np.array([lib().or_spin_colour(L, i) for i in range(8 * L * L)], np.int32)


def energy(L, J, s):
    return int(lib().or_energy(L, np.ascontiguousarray(J, np.int8), np.ascontiguousarray(s, np.int8)))


def metropolis_thresholds(betas, kmax=KMAX):
    """[n_temps][kmax + 1]: floor(exp(-2 k beta) 2^32), k = 1..kmax (entry 0 unused)."""
    betas = np.ascontiguousarray(betas, np.float64)
    thr = np.zeros((len(betas), kmax + 1), np.uint32)
    lib().or_metropolis_thresholds(len(betas), betas, int(kmax), thr)
    return thr


def coupler_kmax(L, J):
    """Largest sum of |J| over one spin's couplers."""
    return int(lib().or_coupler_kmax(L, np.ascontiguousarray(J, np.int8)))


def exchange_thresholds(betas):
    """Returns (off, table): pair p owns table[off[p]:off[p+1]] for h = 1..H_p."""
    betas = np.ascontiguousarray(betas, np.float64)
    nt = len(betas)
    total = lib().or_exchange_thresholds(nt, betas, None, None)
    if total < 0:
        raise ValueError("beta ladder must be strictly descending")
    off = np.zeros(max(nt, 1), np.int64)
    table = np.zeros(max(total, 1), np.uint32)
    lib().or_exchange_thresholds(nt, betas, off.ctypes.data, table.ctypes.data)
    return off, table[:total]


class PTState:
    """Oracle PT state for one instance: R runs x N_T slots, configurations in slot order."""

    def __init__(self, L, J, betas, n_runs, seed, uid, spins=None, walk=False):
        self.L = L
        self.N = 8 * L * L
        self.J = np.ascontiguousarray(J, np.int8).copy()
        self.betas = np.ascontiguousarray(betas, np.float64).copy()
        self.NT = len(self.betas)
        self.R = n_runs
        self.seed = _u32(seed)
        self.uid = _u32(uid)
        self.spins = np.zeros((self.R, self.NT, self.N), np.int8)
        if spins is None:
            lib().or_pt_init_spins(L, self.NT, self.R, self.seed, self.uid, self.spins)
        else:
            self.spins[...] = np.asarray(spins, np.int8).reshape(self.R, self.NT, self.N)
        self.E = np.zeros((self.R, self.NT), np.int32)
        self.best = np.zeros(self.R, np.int32)
        self.first = np.zeros(self.R, np.int32)
        self.macc = np.zeros((self.R, self.NT), np.uint64)
        self.xacc = np.zeros((self.R, max(self.NT - 1, 1)), np.uint64)
        self.sweep = 0
        lib().or_pt_start(L, self.J, self.NT, self.R, self.spins, self.E, self.best, self.first)
        # temperature random walk (Sec. III.B): copy[r, t] = copy whose configuration
        # is in slot t (copies are named by their starting slot); hot / trips by copy
        self.walk = bool(walk)
        if self.walk:
            self.copy = np.tile(np.arange(self.NT, dtype=np.int32), (self.R, 1))
            self.hot = np.zeros((self.R, self.NT), np.uint64)
            self.trips = np.zeros((self.R, self.NT), np.uint64)
            self.wstate = np.zeros((self.R, self.NT), np.uint8)
            self.n_passes = 0

    def sweeps(self, n, exchange_every=1):
        args = (self.L, self.J, self.NT, self.betas, self.R, self.seed, self.uid, self.spins, self.E,
                self.best, self.first, self.macc, self.xacc, self.sweep, int(n), int(exchange_every))
        if self.walk:
            rc = lib().or_pt_sweeps_walk(*args, self.copy, self.hot, self.trips, self.wstate)
            if exchange_every > 0 and self.NT > 1:
                self.n_passes += (self.sweep + int(n)) // exchange_every - self.sweep // exchange_every
        else:
            rc = lib().or_pt_sweeps(*args)
        if rc:
            raise ValueError("oracle sweep failed (bad ladder)")
        self.sweep += int(n)

    def exchange(self):
        args = (self.L, self.J, self.NT, self.betas, self.R, self.seed, self.uid, self.spins, self.E,
                self.xacc, self.sweep)
        if self.walk:
            rc = lib().or_pt_exchange_walk(*args, self.copy, self.hot, self.trips, self.wstate)
            self.n_passes += 1 if self.NT > 1 else 0
        else:
            rc = lib().or_pt_exchange(*args)
        if rc:
            raise ValueError("oracle exchange failed (bad ladder)")

    def full_energies(self):
        return np.array([[energy(self.L, self.J, self.spins[r, t]) for t in range(self.NT)]
                         for r in range(self.R)], np.int32)

    def tts(self, target=TARGET_BEST, horizon=None):
        return tts(self.best, self.first, target, self.sweep if horizon is None else horizon)


def tts(best, first, target=TARGET_BEST, horizon=2**31 - 2):
    best = np.ascontiguousarray(best, np.int32)
    first = np.ascontiguousarray(first, np.int32)
    t, h, tg = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    lib().or_tts(len(best), best, first, int(target), int(horizon),
                 ctypes.byref(t), ctypes.byref(h), ctypes.byref(tg))
    return t.value, h.value, tg.value


def tts_eval(L, J, betas, n_runs, seed, uid, S, pass_mult=1, exchange_every=1):
    t, h, tg = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    rc = lib().or_tts_eval(L, np.ascontiguousarray(J, np.int8), len(betas),
                           np.ascontiguousarray(betas, np.float64), n_runs, _u32(seed), _u32(uid),
                           int(S), int(pass_mult), int(exchange_every),
                           ctypes.byref(t), ctypes.byref(h), ctypes.byref(tg))
    if rc:
        raise ValueError("oracle TTS evaluation failed (bad ladder)")
    return t.value, h.value, tg.value


def tts_eval_doubling(L, J, betas, n_runs, seed, uid, S0, Smax, exchange_every=1):
    """(tts, n_hit, target, level) under the doubling budget S0, 2 S0, ... Smax."""
    t, h, tg, lv = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    rc = lib().or_tts_eval_doubling(L, np.ascontiguousarray(J, np.int8), len(betas),
                                    np.ascontiguousarray(betas, np.float64), n_runs, _u32(seed), _u32(uid),
                                    int(S0), int(Smax), int(exchange_every),
                                    ctypes.byref(t), ctypes.byref(h), ctypes.byref(tg), ctypes.byref(lv))
    if rc:
        raise ValueError("oracle TTS evaluation failed (bad ladder)")
    return t.value, h.value, tg.value, lv.value


def engineer_draw(L, J, seed, base_uid, step, proposal=0):
    e, v = ctypes.c_int32(), ctypes.c_int32()
    cu, ua = ctypes.c_uint32(), ctypes.c_uint32()
    lib().or_engineer_draw(L, np.ascontiguousarray(J, np.int8), _u32(seed), _u32(base_uid),
                           _u32(step), _u32(proposal), ctypes.byref(e), ctypes.byref(v),
                           ctypes.byref(cu), ctypes.byref(ua))
    return e.value, v.value, cu.value, ua.value


def rao_accept(tts_cur, tts_new, direction=1, beta_rao=-1.0, u=0):
    """Algorithm 1's decision for one candidate (beta_rao < 0: greedy)."""
    return bool(lib().or_rao_accept(int(tts_cur), int(tts_new), int(direction), float(beta_rao), _u32(u)))


def engineer_run(L, J, betas, n_runs, seed, base_uid, S, pass_mult, exchange_every,
                 step0, n_steps, beta_rao=-1.0, direction=1, tts_cur=-1, max_sweeps=0):
    """Returns (J_final, tts_final, log) with log a dict of per-step arrays.
    max_sweeps > 0: every evaluation uses the doubling budget S .. max_sweeps."""
    J = np.ascontiguousarray(J, np.int8).copy()
    cur = ctypes.c_int32(int(tts_cur))
    logs = {k: np.zeros(max(n_steps, 1), np.int32) for k in ("edge", "old", "new", "tts", "accept")}
    rc = lib().or_engineer_run_budget(L, J, len(betas), np.ascontiguousarray(betas, np.float64), n_runs,
                                      _u32(seed), _u32(base_uid), int(S), int(pass_mult), int(max_sweeps),
                                      int(exchange_every), _u32(step0), int(n_steps), float(beta_rao),
                                      int(direction), ctypes.byref(cur),
                                      *(logs[k].ctypes.data for k in ("edge", "old", "new", "tts", "accept")))
    if rc:
        raise ValueError("oracle engineering failed")
    return J, cur.value, {k: v[:n_steps] for k, v in logs.items()}


def engineer_run_adaptive(L, J, betas, seed, base_uid, S, pass_mult, exchange_every, step0, n_steps,
                          n0, n_min, cost_max, tts_cur, beta_rao=-1.0, beta_per_run=0.0, direction=1,
                          max_sweeps=0):
    """RAO with Appendix B's adaptive budget (see or_engineer_run_adaptive):
    returns (J_final, tts_final, n_after, log) with per-step edge, new, tts,
    accept, n (runs used) and level (sweeps used)."""
    J = np.ascontiguousarray(J, np.int8).copy()
    cur, n = ctypes.c_int32(int(tts_cur)), ctypes.c_int32(int(n0))
    keys = ("edge", "new", "tts", "accept", "n", "level")
    logs = {k: np.zeros(max(n_steps, 1), np.int32) for k in keys}
    rc = lib().or_engineer_run_adaptive(L, J, len(betas), np.ascontiguousarray(betas, np.float64), _u32(seed),
                                        _u32(base_uid), int(S), int(pass_mult), int(max_sweeps), int(exchange_every),
                                        _u32(step0), int(n_steps), float(beta_rao), float(beta_per_run),
                                        int(direction), int(n_min), int(cost_max), ctypes.byref(n),
                                        ctypes.byref(cur), *(logs[k].ctypes.data for k in keys))
    if rc:
        raise ValueError("oracle engineering failed")
    return J, cur.value, n.value, {k: v[:n_steps] for k, v in logs.items()}


def ground_energy_bipartite(L, J):
    return int(lib().or_ground_energy_bipartite(L, np.ascontiguousarray(J, np.int8)))


# --------------------------------------------------------------------------
# Planted-solution instances and loop adaptive optimisation (Sec. IV,
# Algorithm 2); definitions of the draws in pt_oracle.c.
LOOP_WORDS = 9


def lao_plant(L, seed, uid, n_loops, w_max=5):
    """(planted spins [N], loops [n_loops][9], couplers [E], E_GS)."""
    N, E = 8 * L * L, 16 * L * L + 8 * L * (L - 1)
    planted = np.zeros(N, np.int8)
    loops = np.zeros((n_loops, LOOP_WORDS), np.int32)
    J = np.zeros(E, np.int8)
    eg = ctypes.c_int32()
    if lib().or_lao_plant(L, _u32(seed), _u32(uid), int(n_loops), int(w_max), planted, loops, J, ctypes.byref(eg)):
        raise ValueError("no admissible loop found")
    return planted, loops, J, eg.value


class LAOState:
    """Oracle loop adaptive optimisation on one planted instance."""

    def __init__(self, L, betas, n_runs, seed, uid, n_loops, w_max=5, S=1024, exchange_every=1,
                 beta_rao=-1.0, direction=1):
        self.L, self.betas, self.R, self.seed, self.uid = L, np.ascontiguousarray(betas, np.float64), n_runs, seed, uid
        self.M, self.w_max, self.S, self.x, self.beta, self.direction = n_loops, w_max, S, exchange_every, beta_rao, direction
        self.planted, self.loops, self.J, self.E_gs = lao_plant(L, seed, uid, n_loops, w_max)
        self.tts = -1

    def run(self, step0, n_steps):
        eg, tc = ctypes.c_int32(self.E_gs), ctypes.c_int32(self.tts)
        logs = [np.zeros(max(n_steps, 1), np.int32) for _ in range(4)]
        rc = lib().or_lao_run(self.L, len(self.betas), self.betas, self.R, _u32(self.seed), _u32(self.uid), self.M,
                              self.w_max, int(self.S), int(self.x), float(self.beta), int(self.direction),
                              _u32(step0), int(n_steps), self.planted, self.loops, self.J, ctypes.byref(eg),
                              ctypes.byref(tc), *logs)
        if rc:
            raise ValueError("oracle LAO failed")
        self.E_gs, self.tts = eg.value, tc.value
        return {"removed": logs[0][:n_steps], "tts": logs[1][:n_steps], "E_gs": logs[2][:n_steps],
                "accepted": logs[3][:n_steps]}


def overlaps(spins, E, E_gs):
    """Ground / first-excited overlaps (Sec. III.B) of PT replicas: spins
    [R][N_T][N] (+-1, slot order), energies E [R][N_T].  The first excited level
    is the lowest replica energy above E_gs; samples: per run, its coldest
    replica at E_gs (ground) and its coldest replica at that level (excited);
    overlap |1 - 2 h / N| for Hamming distance h; lower medians over the
    distinct ground pairs and over all (ground, excited) pairs (-1 without a
    pair)."""
    spins = np.asarray(spins)
    E = np.asarray(E)
    R, NT, N = spins.shape
    above = [int(e) for e in E.ravel() if e > E_gs]
    E1 = min(above) if above else 2**31 - 1

    def pick(level):
        out = []
        for r in range(R):
            for t in range(NT):
                if E[r, t] == level:
                    out.append(spins[r, t])
                    break
        return out

    gs, es = pick(E_gs), pick(E1)

    def q(a, b):
        return abs(N - 2 * int(np.sum(a != b)))

    def lower_median(v):
        if not v:
            return -1
        v = sorted(v)
        return v[(len(v) + 1) // 2 - 1]

    a = [q(gs[i], gs[j]) for i in range(len(gs)) for j in range(i + 1, len(gs))]
    b = [q(x, y) for x in gs for y in es]
    ma, mb = lower_median(a), lower_median(b)
    return dict(n_gs=len(gs), n_es=len(es), E1=E1, q_gs_gs=-1.0 if ma < 0 else ma / N,
                q_gs_es=-1.0 if mb < 0 else mb / N)
