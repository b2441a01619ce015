"""ctypes binding of ``libpt_gb300.so`` (the C ABI declared in include/pt.h).

Argument marshalling only: every step of the PT path runs in the library's
CUDA kernels.  There is no CPU fallback; loading fails loudly when the library
has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpt_gb300.so")
# PT_GB300_DEBUG=1 selects the build with device-side bounds checks
# (pt_debug_enabled / pt_debug_status); it is built by build.build(debug=True).
DEBUG_LIB_PATH = os.path.join(_HERE, "libpt_gb300_debug.so")
if os.environ.get("PT_GB300_DEBUG", "") not in ("", "0"):
    LIB_PATH = DEBUG_LIB_PATH

PT_OK, PT_ERR_ARG, PT_ERR_CUDA, PT_ERR_TIMEOUT, PT_ERR_OOM, PT_ERR_STATE = range(6)
PT_TARGET_BEST = 2**31 - 1
PT_KMAX = 18

_ERRNAMES = {1: "PT_ERR_ARG", 2: "PT_ERR_CUDA", 3: "PT_ERR_TIMEOUT", 4: "PT_ERR_OOM", 5: "PT_ERR_STATE"}


class PTError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class pt_rule(C.Structure):
    _fields_ = [("S", C.c_int32), ("pass_mult", C.c_int32), ("exchange_every", C.c_int32),
                ("direction", C.c_int32), ("beta_rao", C.c_double), ("max_sweeps", C.c_int32)]


class pt_graph(C.Structure):
    _fields_ = [("n", C.c_int32), ("n_edges", C.c_int32), ("ei", C.c_void_p), ("ej", C.c_void_p),
                ("chimera_L", C.c_int32)]


class pt_step_result(C.Structure):
    _fields_ = [("edge", C.c_int32), ("old_value", C.c_int32), ("new_value", C.c_int32),
                ("tts_old", C.c_int32), ("tts_new", C.c_int32), ("accepted", C.c_int32),
                ("cand_uid", C.c_uint32), ("n_runs", C.c_int32), ("level", C.c_int32)]


PT_LOOP_WORDS = 9


class pt_lao_result(C.Structure):
    _fields_ = [("removed", C.c_int32), ("loop", C.c_int32 * PT_LOOP_WORDS), ("E_gs_new", C.c_int32),
                ("tts_old", C.c_int32), ("tts_new", C.c_int32), ("accepted", C.c_int32), ("cand_uid", C.c_uint32)]


# (name, restype, argtypes) of every entry point declared in include/pt.h
_VP = C.c_void_p
_I32P = C.POINTER(C.c_int32)
SIGNATURES = [
    ("pt_last_error", C.c_char_p, [_VP]),
    ("pt_create", C.c_int, [C.POINTER(_VP), C.c_int32, _VP, C.c_int32, _VP, C.c_int32, C.c_int32,
                            C.c_uint32, C.c_uint32, _VP]),
    ("pt_destroy", None, [_VP]),
    ("pt_reset", C.c_int, [_VP, C.c_uint32]),
    ("pt_set_spins", C.c_int, [_VP, _VP]),
    ("pt_sweep", C.c_int, [_VP, C.c_int32, C.c_int32]),
    ("pt_exchange", C.c_int, [_VP]),
    ("pt_get_state", C.c_int, [_VP] + [_VP] * 8),
    ("pt_tts", C.c_int, [_VP, C.c_int32, C.c_int32, _I32P, _I32P, _I32P]),
    ("pt_tts_eval", C.c_int, [_VP, C.c_uint32, C.c_int32, C.c_int32, C.c_int32, _I32P, _I32P, _I32P]),
    ("pt_tts_eval_many", C.c_int, [_VP, C.c_int32, _VP, _VP, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                   _VP, _VP, _VP, _VP]),
    ("pt_tts_eval_doubling", C.c_int, [_VP, C.c_uint32, C.c_int32, C.c_int32, C.c_int32, _I32P, _I32P, _I32P,
                                       _I32P]),
    ("pt_set_coupler", C.c_int, [_VP, C.c_int32, C.c_int8]),
    ("pt_get_couplers", C.c_int, [_VP, _VP]),
    ("pt_get_tables", C.c_int, [_VP, _VP, _VP, _VP, C.c_int64, C.POINTER(C.c_int64)]),
    ("pt_get_table_rows", C.c_int, [_VP, _I32P]),
    ("engineer_begin", C.c_int, [_VP, C.POINTER(pt_rule), C.c_uint32, _I32P]),
    ("engineer_step", C.c_int, [_VP, C.c_uint32, C.POINTER(pt_step_result)]),
    ("engineer_run", C.c_int, [_VP, C.c_uint32, C.c_int32, C.c_int32, C.POINTER(pt_step_result)]),
    ("lao_plant", C.c_int, [C.c_int32, C.c_uint32, C.c_uint32, C.c_int32, C.c_int32, _VP, _VP, _VP, _I32P]),
    ("lao_begin", C.c_int, [_VP, C.POINTER(pt_rule), C.c_uint32, C.c_int32, C.c_int32, _I32P]),
    ("lao_run", C.c_int, [_VP, C.c_uint32, C.c_int32, C.c_int32, C.POINTER(pt_lao_result)]),
    ("lao_state", C.c_int, [_VP, _VP, _VP, _VP, _I32P, _I32P]),
    ("pt_overlaps", C.c_int, [_VP, C.c_int32, _I32P, _I32P, _I32P, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("engineer_current_tts", C.c_int, [_VP, _I32P]),
    ("pt_create_graph", C.c_int, [C.POINTER(_VP), C.POINTER(pt_graph), _VP, _VP, C.c_int32, C.c_int32, C.c_uint32,
                                  C.c_uint32, _VP]),
    ("engineer_current_state", C.c_int, [_VP, _I32P, _I32P]),
    ("engineer_set_adaptive", C.c_int, [_VP, C.c_int32, C.c_int32, C.c_int64, C.c_double]),
    ("engineer_adaptive_runs", C.c_int, [_VP, _I32P]),
    ("pt_checkpoint", C.c_int, [_VP, _VP, C.POINTER(C.c_size_t)]),
    ("pt_restore", C.c_int, [_VP, _VP, C.c_size_t]),
    ("pt_set_schedule", C.c_int, [_VP, C.c_int32, C.c_int32, C.c_int32]),
    ("pt_get_schedule", C.c_int, [_VP, _I32P, _I32P, _I32P]),
    ("pt_autotune", C.c_int, [_VP, C.c_int32, C.c_int32]),
    ("pt_set_mapping", C.c_int, [_VP, C.c_int32, C.c_int32, C.c_int32]),
    ("pt_get_mapping", C.c_int, [_VP, _I32P]),
    ("pt_set_walk_stats", C.c_int, [_VP, C.c_int32]),
    ("pt_get_walk_stats", C.c_int, [_VP, _VP, _VP, C.POINTER(C.c_uint64)]),
    ("pt_launch_count", C.c_uint64, [_VP]),
    ("pt_select_device", C.c_int, [C.c_int32]),
    ("pt_set_timing", C.c_int, [_VP, C.c_int]),
    ("pt_last_sweep_timing", C.c_int, [_VP, C.POINTER(C.c_double), _I32P]),
    ("pt_sweep_timing_total", C.c_int, [_VP, C.POINTER(C.c_double), C.POINTER(C.c_uint64)]),
    ("pt_eval_stats", C.c_int, [_VP, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64),
                                C.POINTER(C.c_double), C.c_int]),
    ("pt_int_issue_rate", C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_double),
                                    C.POINTER(C.c_double), _VP]),
    ("pt_tts_eval_noalloc", C.c_int, [C.c_int32, _VP, C.c_int32, _VP, C.c_int32, C.c_int32,
                                      C.c_uint32, C.c_uint32, C.c_int32, C.c_int32, C.c_int32, _VP,
                                      _I32P, _I32P, _I32P]),
    ("pt_batch_last_error", C.c_char_p, [_VP]),
    ("pt_batch_create", C.c_int, [C.POINTER(_VP), C.c_int32, _VP, C.c_int32, C.c_uint32, _VP]),
    ("pt_batch_destroy", None, [_VP]),
    ("pt_batch_reset", C.c_int, [_VP]),
    ("pt_batch_run", C.c_int, [_VP, C.c_int32, C.c_int32]),
    ("pt_batch_tts", C.c_int, [_VP, C.c_int32, _VP, _VP, _VP]),
    ("pt_batch_get_state", C.c_int, [_VP, C.c_int32] + [_VP] * 6),
    ("pt_batch_set_schedule", C.c_int, [_VP, C.c_int32, C.c_int32, C.c_int32, C.c_int32]),
    ("pt_batch_get_schedule", C.c_int, [_VP, C.c_int32, _I32P, _I32P, _I32P]),
    ("pt_batch_set_mapping", C.c_int, [_VP, C.c_int32, C.c_int32, C.c_int32, C.c_int32]),
    ("pt_batch_get_mapping", C.c_int, [_VP, C.c_int32, _I32P]),
    ("pt_batch_autotune", C.c_int, [_VP, C.c_int32, _I32P]),
    ("pt_batch_info", C.c_int, [_VP, C.POINTER(C.c_double), _I32P, _I32P, _I32P, C.POINTER(C.c_uint64)]),
    ("sg_last_error", C.c_char_p, [_VP]),
    ("sg_create", C.c_int, [C.POINTER(_VP), C.c_int32, C.c_int32, _VP]),
    ("sg_destroy", None, [_VP]),
    ("sg_num_params", C.c_int64, [_VP]),
    ("sg_set_params", C.c_int, [_VP, _VP]),
    ("sg_get_params", C.c_int, [_VP, _VP]),
    ("sg_forward", C.c_int, [_VP, C.c_int32, C.c_int32, _VP, _VP]),
    ("sg_grad", C.c_int, [_VP, C.c_int32, C.c_int32, _VP, _VP, C.POINTER(C.c_float), _VP]),
    ("sg_adam", C.c_int, [_VP, C.c_float]),
    ("sg_train_step", C.c_int, [_VP, C.c_int32, C.c_int32, _VP, _VP, C.c_float, C.POINTER(C.c_float)]),
    ("sg_launch_count", C.c_uint64, [_VP]),
    ("engineer_guided_step", C.c_int, [_VP, _VP, C.c_uint32, C.c_int32, C.c_int32,
                                       C.POINTER(pt_step_result), _VP, _VP]),
    ("pt_debug_enabled", C.c_int, []),
    ("pt_debug_status", C.c_int, [C.POINTER(C.c_uint32)]),
]


class pt_instance_desc(C.Structure):
    _fields_ = [("chimera_L", C.c_int32), ("n_temps", C.c_int32), ("J", C.c_void_p),
                ("betas", C.c_void_p), ("uid", C.c_uint32)]

_lib = None


def load():
    """Loads the in-tree library (build it first with paper_1605_03607_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() (no CPU fallback exists)")
        lib = C.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def debug_enabled():
    """True when the loaded library is the bounds-checking debug build."""
    return bool(load().pt_debug_enabled())


def debug_status():
    """First failed device-side bounds check since the last call (0: none)."""
    c = C.c_uint32()
    _check(load().pt_debug_status(C.byref(c)), None)
    return int(c.value)


def select_device(device):
    """Current device of the library's CUDA runtime for this host thread."""
    _check(load().pt_select_device(int(device)), None)


INT_ISSUE_KINDS = ("lop3", "imad", "lop3_imad", "dp4a", "philox_round")


def int_issue_rate(kind, iters=1 << 16, reps=3, stream=None):
    """Measured 32-bit integer operations per second of one instruction kind
    over the whole current device (pt_int_issue_rate); returns (ops_per_s,
    ms_per_launch).  `kind` is an index or a name of INT_ISSUE_KINDS."""
    k = INT_ISSUE_KINDS.index(kind) if isinstance(kind, str) else int(kind)
    ops, ms = C.c_double(), C.c_double()
    _check(load().pt_int_issue_rate(k, int(iters), int(reps), C.byref(ops), C.byref(ms),
                                    None if stream is None else C.c_void_p(stream)), None)
    return ops.value, ms.value


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _check(rc, h=None):
    if rc != PT_OK:
        msg = load().pt_last_error(h)
        raise PTError(rc, msg.decode() if msg else "")


class PTHandle:
    """One instance, n_runs PT runs of len(betas) slots on the GPU (owner of a pt_handle)."""

    def __init__(self, L, J, betas, n_runs, seed, uid, stream=None, edges=None):
        """edges (optional): (ei, ej) coupler list on C_L for J in that order
        (pt_create_graph); missing couplers of C_L are zero."""
        lib = load()
        self.L = int(L)
        self.N = 8 * self.L * self.L
        J = np.ascontiguousarray(J, np.int8)
        betas = np.ascontiguousarray(betas, np.float64)
        self.NT = len(betas)
        self.R = int(n_runs)
        h = C.c_void_p()
        st = None if stream is None else C.c_void_p(stream)
        if edges is None:
            self.n_edges = len(J)
            rc = lib.pt_create(C.byref(h), self.L, _ptr(J), self.n_edges, _ptr(betas), self.NT, self.R,
                               int(seed) & 0xFFFFFFFF, int(uid) & 0xFFFFFFFF, st)
        else:
            ei = np.ascontiguousarray(edges[0], np.int32)
            ej = np.ascontiguousarray(edges[1], np.int32)
            if len(ei) != len(J) or len(ej) != len(J):
                raise ValueError("one coupler value per listed edge")
            g = pt_graph(self.N, len(J), ei.ctypes.data, ej.ctypes.data, self.L)
            self.n_edges = 16 * self.L * self.L + 8 * self.L * (self.L - 1)
            rc = lib.pt_create_graph(C.byref(h), C.byref(g), _ptr(J), _ptr(betas), self.NT, self.R,
                                     int(seed) & 0xFFFFFFFF, int(uid) & 0xFFFFFFFF, st)
        _check(rc, None)
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            load().pt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- PT
    def reset(self, uid):
        _check(load().pt_reset(self.h, int(uid) & 0xFFFFFFFF), self.h)

    def set_spins(self, spins):
        s = np.ascontiguousarray(spins, np.int8).reshape(self.R, self.NT, self.N)
        _check(load().pt_set_spins(self.h, _ptr(s)), self.h)

    def sweep(self, n, exchange_every=1):
        _check(load().pt_sweep(self.h, int(n), int(exchange_every)), self.h)

    def exchange(self):
        _check(load().pt_exchange(self.h), self.h)

    def state(self):
        spins = np.zeros((self.R, self.NT, self.N), np.int8)
        E = np.zeros((self.R, self.NT), np.int32)
        perm = np.zeros((self.R, self.NT), np.uint8)
        best = np.zeros(self.R, np.int32)
        first = np.zeros(self.R, np.int32)
        macc = np.zeros((self.R, self.NT), np.uint64)
        xacc = np.zeros((self.R, max(self.NT - 1, 1)), np.uint64)
        sweep = np.zeros(1, np.uint64)
        _check(load().pt_get_state(self.h, _ptr(spins), _ptr(E), _ptr(perm), _ptr(best), _ptr(first),
                                   _ptr(macc), _ptr(xacc), _ptr(sweep)), self.h)
        return dict(spins=spins, E=E, perm=perm, best=best, first=first, macc=macc, xacc=xacc,
                    sweep=int(sweep[0]))

    def tts(self, target=PT_TARGET_BEST, horizon=None):
        if horizon is None:
            horizon = self.state()["sweep"]
        t, n, tg = C.c_int32(), C.c_int32(), C.c_int32()
        _check(load().pt_tts(self.h, int(target), int(horizon), C.byref(t), C.byref(n), C.byref(tg)), self.h)
        return t.value, n.value, tg.value

    def tts_eval(self, uid, S, pass_mult=1, exchange_every=1):
        t, n, tg = C.c_int32(), C.c_int32(), C.c_int32()
        _check(load().pt_tts_eval(self.h, int(uid) & 0xFFFFFFFF, int(S), int(pass_mult),
                                  int(exchange_every), C.byref(t), C.byref(n), C.byref(tg)), self.h)
        return t.value, n.value, tg.value

    def set_coupler(self, edge, value):
        _check(load().pt_set_coupler(self.h, int(edge), int(value)), self.h)

    def couplers(self):
        J = np.zeros(self.n_edges, np.int8)
        _check(load().pt_get_couplers(self.h, _ptr(J)), self.h)
        return J

    def table_rows(self):
        r = C.c_int32()
        _check(load().pt_get_table_rows(self.h, C.byref(r)), self.h)
        return r.value

    def tables(self):
        n = C.c_int64()
        _check(load().pt_get_tables(self.h, None, None, None, 0, C.byref(n)), self.h)
        thr = np.zeros((self.NT, self.table_rows()), np.uint32)
        xoff = np.zeros(self.NT, np.int64)
        xthr = np.zeros(max(n.value, 1), np.uint32)
        _check(load().pt_get_tables(self.h, _ptr(thr), _ptr(xoff), _ptr(xthr), len(xthr), C.byref(n)), self.h)
        return thr, xoff, xthr[:n.value]

    # -- RAO (Algorithm 1)
    def tts_eval_doubling(self, uid, S0, Smax, exchange_every=1):
        """(tts, n_hit, target, level) under the doubling budget S0, 2 S0, ... Smax."""
        t, h, tg, lv = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        _check(load().pt_tts_eval_doubling(self.h, int(uid) & 0xFFFFFFFF, int(S0), int(Smax), int(exchange_every),
                                           C.byref(t), C.byref(h), C.byref(tg), C.byref(lv)), self.h)
        return t.value, h.value, tg.value, lv.value

    def tts_eval_many(self, J, uids, S, pass_mult=1, max_sweeps=0, exchange_every=1):
        """Batched evaluation of k coupler vectors J [k, n_edges] with PT keys uids:
        dict of k-arrays tts, n_hit, target, level."""
        J = np.ascontiguousarray(J, np.int8).reshape(-1, self.n_edges)
        k = J.shape[0]
        u = np.ascontiguousarray(np.asarray(uids, np.int64) & 0xFFFFFFFF, np.uint32)
        if len(u) != k:
            raise ValueError("one uid per coupler vector")
        out = {n: np.zeros(k, np.int32) for n in ("tts", "n_hit", "target", "level")}
        _check(load().pt_tts_eval_many(self.h, k, _ptr(J), _ptr(u), int(S), int(pass_mult), int(max_sweeps),
                                       int(exchange_every), *(_ptr(out[n]) for n in ("tts", "n_hit", "target",
                                                                                     "level"))), self.h)
        return out

    def engineer_begin(self, S, pass_mult=1, exchange_every=1, base_uid=0, beta_rao=-1.0, direction=1,
                       max_sweeps=0):
        rule = pt_rule(int(S), int(pass_mult), int(exchange_every), int(direction), float(beta_rao),
                       int(max_sweeps))
        t = C.c_int32()
        _check(load().engineer_begin(self.h, C.byref(rule), int(base_uid) & 0xFFFFFFFF, C.byref(t)), self.h)
        return t.value

    def engineer_run(self, step0, n_steps, speculation=1, log=None):
        """n_steps RAO steps from step0.  log (path or writable text file, optional):
        one JSON record per step appended (see _log_steps)."""
        out = (pt_step_result * max(n_steps, 1))()
        e0 = self.eval_stats() if log is not None else None
        _check(load().engineer_run(self.h, int(step0) & 0xFFFFFFFF, int(n_steps), int(speculation), out), self.h)
        keys = ("edge", "old_value", "new_value", "tts_old", "tts_new", "accepted", "cand_uid", "n_runs", "level")
        res = {k: np.array([getattr(out[i], k) for i in range(n_steps)], np.int64) for k in keys}
        if log is not None:
            _log_steps(log, "rao", step0, res, e0, self.eval_stats(), self.engineer_state()[1])
        return res

    def set_adaptive(self, n0, n_min=16, cost_max=1 << 40, beta_per_run=0.0):
        """Appendix B's adaptive budget for engineer_run (n0 = 0: off)."""
        _check(load().engineer_set_adaptive(self.h, int(n0), int(n_min), int(cost_max), float(beta_per_run)), self.h)

    def adaptive_runs(self):
        n = C.c_int32()
        _check(load().engineer_adaptive_runs(self.h, C.byref(n)), self.h)
        return n.value

    def engineer_step(self, step):
        return self.engineer_run(step, 1, 1)

    def lao_begin(self, S, uid, n_loops, w_max=5, exchange_every=1, beta_rao=-1.0, direction=1):
        """Planted instance with n_loops loops (Algorithm 2); returns its TTS against E_GS."""
        rule = pt_rule(int(S), 1, int(exchange_every), int(direction), float(beta_rao), 0)
        t = C.c_int32()
        _check(load().lao_begin(self.h, C.byref(rule), int(uid) & 0xFFFFFFFF, int(n_loops), int(w_max), C.byref(t)),
               self.h)
        self.n_loops = int(n_loops)
        return t.value

    def lao_run(self, step0, n_steps, speculation=1, log=None):
        """n_steps LAO steps from step0 (>= 1); log as in engineer_run."""
        out = (pt_lao_result * max(n_steps, 1))()
        e0 = self.eval_stats() if log is not None else None
        _check(load().lao_run(self.h, int(step0) & 0xFFFFFFFF, int(n_steps), int(speculation), out), self.h)
        keys = ("removed", "E_gs_new", "tts_old", "tts_new", "accepted", "cand_uid")
        res = {k: np.array([getattr(out[i], k) for i in range(n_steps)], np.int64) for k in keys}
        res["loop"] = np.array([list(out[i].loop) for i in range(n_steps)], np.int32).reshape(n_steps, PT_LOOP_WORDS)
        if log is not None:
            _log_steps(log, "lao", step0, res, e0, self.eval_stats(), self.engineer_state()[1])
        return res

    def overlaps(self, E_gs):
        """Ground / first-excited overlaps of the runs' coldest-slot configurations:
        dict(n_gs, n_es, E1, q_gs_gs, q_gs_es)."""
        a, b, e1 = C.c_int32(), C.c_int32(), C.c_int32()
        qa, qb = C.c_double(), C.c_double()
        _check(load().pt_overlaps(self.h, int(E_gs), C.byref(a), C.byref(b), C.byref(e1), C.byref(qa), C.byref(qb)),
               self.h)
        return dict(n_gs=a.value, n_es=b.value, E1=e1.value, q_gs_gs=qa.value, q_gs_es=qb.value)

    def lao_state(self):
        planted = np.zeros(self.N, np.int8)
        loops = np.zeros((self.n_loops, PT_LOOP_WORDS), np.int32)
        J = np.zeros(self.n_edges, np.int8)
        eg, t = C.c_int32(), C.c_int32()
        _check(load().lao_state(self.h, _ptr(planted), _ptr(loops), _ptr(J), C.byref(eg), C.byref(t)), self.h)
        return dict(planted=planted, loops=loops, J=J, E_gs=eg.value, tts=t.value)

    def engineer_guided_step(self, model, step, n_prop=64, top=4):
        """One best-of-top step; returns (results in rank order, predictions, ranked indices).
        model None: no ranking, proposals 0..top-1 are evaluated (the plain
        loop under the same acceptance rule)."""
        out = (pt_step_result * top)()
        pred = np.zeros(n_prop, np.float32)
        ranked = np.zeros(top, np.int32)
        _check(load().engineer_guided_step(self.h, None if model is None else model.m, int(step) & 0xFFFFFFFF,
                                           int(n_prop), int(top), out, _ptr(pred), _ptr(ranked)), self.h)
        keys = ("edge", "old_value", "new_value", "tts_old", "tts_new", "accepted", "cand_uid", "n_runs", "level")
        res = {k: np.array([getattr(out[i], k) for i in range(top)], np.int64) for k in keys}
        return res, pred, ranked

    def engineer_tts(self):
        t = C.c_int32()
        _check(load().engineer_current_tts(self.h, C.byref(t)), self.h)
        return t.value

    def engineer_state(self):
        """(TTS, runs that hit the target) of the loop's current instance."""
        t, n = C.c_int32(), C.c_int32()
        _check(load().engineer_current_state(self.h, C.byref(t), C.byref(n)), self.h)
        return t.value, n.value

    # -- checkpoint / schedule / accounting
    def checkpoint(self):
        n = C.c_size_t()
        _check(load().pt_checkpoint(self.h, None, C.byref(n)), self.h)
        buf = np.zeros(n.value, np.uint8)
        _check(load().pt_checkpoint(self.h, _ptr(buf), C.byref(n)), self.h)
        return buf

    def restore(self, buf):
        buf = np.ascontiguousarray(buf, np.uint8)
        _check(load().pt_restore(self.h, _ptr(buf), len(buf)), self.h)

    def set_schedule(self, slot_parallel=0, runs_per_cta=0, sweeps_per_launch=0):
        _check(load().pt_set_schedule(self.h, int(slot_parallel), int(runs_per_cta), int(sweeps_per_launch)), self.h)

    def autotune(self, n_inst=16, trial_sweeps=64):
        _check(load().pt_autotune(self.h, int(n_inst), int(trial_sweeps)), self.h)
        return self.schedule()

    def set_mapping(self, team, slot_parallel=0, runs_per_cta=0):
        _check(load().pt_set_mapping(self.h, int(team), int(slot_parallel), int(runs_per_cta)), self.h)

    def mapping(self):
        t = C.c_int32()
        _check(load().pt_get_mapping(self.h, C.byref(t)), self.h)
        return t.value

    def set_walk_stats(self, on=True):
        _check(load().pt_set_walk_stats(self.h, 1 if on else 0), self.h)

    def walk_stats(self):
        """(hot, trips, n_passes): per run and copy, exchange passes spent in the
        hot half and completed cold -> hot -> cold round trips."""
        hot = np.zeros((self.R, self.NT), np.uint64)
        trips = np.zeros((self.R, self.NT), np.uint64)
        n = C.c_uint64()
        _check(load().pt_get_walk_stats(self.h, _ptr(hot), _ptr(trips), C.byref(n)), self.h)
        return hot, trips, int(n.value)

    def schedule(self):
        a, b, c = C.c_int32(), C.c_int32(), C.c_int32()
        _check(load().pt_get_schedule(self.h, C.byref(a), C.byref(b), C.byref(c)), self.h)
        return a.value, b.value, c.value

    def launch_count(self):
        return int(load().pt_launch_count(self.h))

    def set_timing(self, on=True):
        _check(load().pt_set_timing(self.h, 1 if on else 0), self.h)

    def sweep_timing_total(self):
        ms, n = C.c_double(), C.c_uint64()
        _check(load().pt_sweep_timing_total(self.h, C.byref(ms), C.byref(n)), self.h)
        return ms.value, int(n.value)

    def eval_stats(self, reset=False):
        e, b, ms = C.c_uint64(), C.c_uint64(), C.c_double()
        _check(load().pt_eval_stats(self.h, C.byref(e), C.byref(b), C.byref(ms), 1 if reset else 0), self.h)
        return int(e.value), int(b.value), ms.value

    def last_sweep_timing(self):
        ms, n = C.c_double(), C.c_int32()
        _check(load().pt_last_sweep_timing(self.h, C.byref(ms), C.byref(n)), self.h)
        return ms.value, n.value


def _log_steps(log, kind, step0, res, before, after, hits_now):
    """Appends one JSON line per step of an engineering call: step, the move
    (coupler and old/new value for RAO, removed loop and new ground-state
    energy for LAO), TTS before and after, acceptance, the candidate's PT key,
    and the device time of the call's evaluations divided by the candidates
    evaluated (speculative candidates that were discarded included).  The
    last line of a call also carries the current instance's hit count."""
    import json
    evals = after[0] - before[0]
    ms_per_eval = (after[2] - before[2]) / evals if evals > 0 else None
    n = len(res["tts_new"])
    recs = []
    for i in range(n):
        r = {"kind": kind, "step": int(step0) + i, "tts_old": int(res["tts_old"][i]),
             "tts_new": int(res["tts_new"][i]), "accepted": bool(res["accepted"][i]),
             "cand_uid": int(res["cand_uid"][i]), "device_ms_per_eval": ms_per_eval}
        if kind == "rao":
            r.update(coupler=int(res["edge"][i]), J_old=int(res["old_value"][i]), J_new=int(res["new_value"][i]),
                     runs=int(res["n_runs"][i]), sweeps=int(res["level"][i]))
        else:
            r.update(removed_loop=int(res["removed"][i]), E_gs_new=int(res["E_gs_new"][i]))
        if i == n - 1:
            r.update(call_evals=int(evals), call_batches=int(after[1] - before[1]), n_hit_now=int(hits_now))
        recs.append(json.dumps(r))
    text = "".join(x + "\n" for x in recs)
    if hasattr(log, "write"):
        log.write(text)
    else:
        with open(log, "a") as f:
            f.write(text)


def _check_batch(rc, b=None):
    if rc != PT_OK:
        msg = load().pt_batch_last_error(b)
        raise PTError(rc, msg.decode() if msg else "")


class PTBatch:
    """Many instances (list of dicts with L, J, betas, uid) x n_runs PT runs in one persistent launch."""

    def __init__(self, instances, n_runs, seed, stream=None):
        lib = load()
        self.inst = [dict(L=int(x["L"]), J=np.ascontiguousarray(x["J"], np.int8),
                          betas=np.ascontiguousarray(x["betas"], np.float64), uid=int(x["uid"]))
                     for x in instances]
        self.R = int(n_runs)
        descs = (pt_instance_desc * len(self.inst))()
        for d, x in zip(descs, self.inst):
            d.chimera_L = x["L"]
            d.n_temps = len(x["betas"])
            d.J = x["J"].ctypes.data
            d.betas = x["betas"].ctypes.data
            d.uid = x["uid"] & 0xFFFFFFFF
        b = C.c_void_p()
        rc = lib.pt_batch_create(C.byref(b), len(self.inst), descs, self.R, int(seed) & 0xFFFFFFFF,
                                 None if stream is None else C.c_void_p(stream))
        _check_batch(rc, None)
        self.b = b

    def close(self):
        if getattr(self, "b", None):
            load().pt_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def reset(self):
        _check_batch(load().pt_batch_reset(self.b), self.b)

    def run(self, n_sweeps, exchange_every=1):
        _check_batch(load().pt_batch_run(self.b, int(n_sweeps), int(exchange_every)), self.b)

    def tts(self, horizon):
        n = len(self.inst)
        t, h, tg = (np.zeros(n, np.int32) for _ in range(3))
        _check_batch(load().pt_batch_tts(self.b, int(horizon), _ptr(t), _ptr(h), _ptr(tg)), self.b)
        return t, h, tg

    def state(self, i):
        x = self.inst[i]
        NT, N = len(x["betas"]), 8 * x["L"] ** 2
        spins = np.zeros((self.R, NT, N), np.int8)
        E = np.zeros((self.R, NT), np.int32)
        best = np.zeros(self.R, np.int32)
        first = np.zeros(self.R, np.int32)
        macc = np.zeros((self.R, NT), np.uint64)
        xacc = np.zeros((self.R, max(NT - 1, 1)), np.uint64)
        _check_batch(load().pt_batch_get_state(self.b, int(i), _ptr(spins), _ptr(E), _ptr(best), _ptr(first),
                                               _ptr(macc), _ptr(xacc)), self.b)
        return dict(spins=spins, E=E, best=best, first=first, macc=macc, xacc=xacc)

    def set_schedule(self, block=0, L=0, slot_parallel=0, runs_per_cta=0):
        _check_batch(load().pt_batch_set_schedule(self.b, int(block), int(L), int(slot_parallel),
                                                  int(runs_per_cta)), self.b)

    def schedule(self, L):
        a, b_, c = C.c_int32(), C.c_int32(), C.c_int32()
        _check_batch(load().pt_batch_get_schedule(self.b, int(L), C.byref(a), C.byref(b_), C.byref(c)), self.b)
        return a.value, b_.value, c.value

    def set_mapping(self, team, L=0, slot_parallel=0, runs_per_cta=0):
        _check_batch(load().pt_batch_set_mapping(self.b, int(L), int(team), int(slot_parallel),
                                                 int(runs_per_cta)), self.b)

    def mapping(self, L):
        t = C.c_int32()
        _check_batch(load().pt_batch_get_mapping(self.b, int(L), C.byref(t)), self.b)
        return t.value

    def autotune(self, trial_sweeps=32):
        blk = C.c_int32()
        _check_batch(load().pt_batch_autotune(self.b, int(trial_sweeps), C.byref(blk)), self.b)
        return blk.value

    def info(self):
        ms, g, bl, nb, la = C.c_double(), C.c_int32(), C.c_int32(), C.c_int32(), C.c_uint64()
        _check_batch(load().pt_batch_info(self.b, C.byref(ms), C.byref(g), C.byref(bl), C.byref(nb),
                                          C.byref(la)), self.b)
        return dict(last_run_ms=ms.value, grid=g.value, block=bl.value, bundles=nb.value, launches=int(la.value))


def _check_sg(rc, m=None):
    if rc != PT_OK:
        msg = load().sg_last_error(m)
        raise PTError(rc, msg.decode() if msg else "")


class Surrogate:
    """The surrogate hardness model (log10 TTS from couplers) on the GPU."""

    def __init__(self, hidden=64, layers=4, stream=None):
        m = C.c_void_p()
        _check_sg(load().sg_create(C.byref(m), int(hidden), int(layers),
                                   None if stream is None else C.c_void_p(stream)), None)
        self.m = m
        self.n = int(load().sg_num_params(m))

    def close(self):
        if getattr(self, "m", None):
            load().sg_destroy(self.m)
            self.m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_params(self, theta):
        th = np.ascontiguousarray(theta, np.float32)
        assert th.size == self.n
        _check_sg(load().sg_set_params(self.m, _ptr(th)), self.m)

    def params(self):
        th = np.zeros(self.n, np.float32)
        _check_sg(load().sg_get_params(self.m, _ptr(th)), self.m)
        return th

    def forward(self, L, J):
        J = np.ascontiguousarray(np.atleast_2d(J), np.int8)
        y = np.zeros(J.shape[0], np.float32)
        _check_sg(load().sg_forward(self.m, int(L), J.shape[0], _ptr(J), _ptr(y)), self.m)
        return y

    def grad(self, L, J, t):
        J = np.ascontiguousarray(np.atleast_2d(J), np.int8)
        t = np.ascontiguousarray(t, np.float32)
        g = np.zeros(self.n, np.float32)
        loss = C.c_float()
        _check_sg(load().sg_grad(self.m, int(L), J.shape[0], _ptr(J), _ptr(t), C.byref(loss), _ptr(g)), self.m)
        return loss.value, g

    def adam(self, lr=1e-3):
        _check_sg(load().sg_adam(self.m, float(lr)), self.m)

    def train_step(self, L, J, t, lr=1e-3):
        J = np.ascontiguousarray(np.atleast_2d(J), np.int8)
        t = np.ascontiguousarray(t, np.float32)
        loss = C.c_float()
        _check_sg(load().sg_train_step(self.m, int(L), J.shape[0], _ptr(J), _ptr(t), float(lr), C.byref(loss)),
                  self.m)
        return loss.value

    def launch_count(self):
        return int(load().sg_launch_count(self.m))


def lao_plant(L, seed, uid, n_loops, w_max=5):
    """Host-side planted instance (no GPU work): (planted, loops, J, E_GS)."""
    N, E = 8 * L * L, 16 * L * L + 8 * L * (L - 1)
    planted = np.zeros(N, np.int8)
    loops = np.zeros((n_loops, PT_LOOP_WORDS), np.int32)
    J = np.zeros(E, np.int8)
    eg = C.c_int32()
    _check(load().lao_plant(int(L), int(seed) & 0xFFFFFFFF, int(uid) & 0xFFFFFFFF, int(n_loops), int(w_max),
                            _ptr(planted), _ptr(loops), _ptr(J), C.byref(eg)), None)
    return planted, loops, J, eg.value
