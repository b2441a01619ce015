"""The C-ABI library builds, loads and exports every symbol include/pt.h declares.

Runs without a GPU: only argument validation paths (which return before any
CUDA call) are exercised.
"""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pt.h")


@pytest.fixture(scope="module")
def P():
    import paper_1605_03607_gb300 as pkg
    from paper_1605_03607_gb300 import build as b
    b.build()
    pkg.load()
    return pkg


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w\s\*]*?\b((?:pt|engineer)_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pt_create", "pt_sweep", "pt_exchange", "pt_tts", "engineer_step", "pt_destroy",
                     "pt_tts_eval", "engineer_run", "pt_checkpoint", "pt_restore"):
        assert required in names


def test_every_declared_symbol_is_exported(P):
    out = subprocess.run(["nm", "-D", "--defined-only", P.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    bound = {name for name, _, _ in P.SIGNATURES}
    for name in declared_functions():
        assert name in exported, name
        assert name in bound, name


def test_library_is_sm103a_only(P):
    # the build passes exactly one -gencode (sm_103a) and links cudart statically
    from paper_1605_03607_gb300 import build as b
    assert b.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    out = subprocess.run(["ldd", P.LIB_PATH], capture_output=True, text=True).stdout
    assert "libcudart" not in out


def _create(P, L=4, J=None, betas=None, nt=None, R=8):
    lib = P.load()
    J = W.random_couplers(L, 1, 0) if J is None else J
    betas = W.beta_ladder(16, 0.1, 3.0) if betas is None else betas
    h = ctypes.c_void_p()
    rc = lib.pt_create(ctypes.byref(h), L, J.ctypes.data_as(ctypes.c_void_p), len(J),
                       betas.ctypes.data_as(ctypes.c_void_p), len(betas) if nt is None else nt, R, 1, 0, None)
    return rc, lib.pt_last_error(None).decode()


def test_argument_validation_without_gpu(P):
    J = W.random_couplers(4, 1, 0)
    assert _create(P, L=0)[0] == 1
    assert _create(P, L=17)[0] == 1
    assert _create(P, J=J[:-1])[0] == 1
    bad = J.copy()
    bad[5] = -128                                   # int8 but outside [-127, 127]
    rc, msg = _create(P, J=bad)
    assert rc == 1 and "coupler" in msg
    big = J.copy()
    big[0:4] = 60                                   # spin 0: four couplers summing to 240 > 127
    rc, msg = _create(P, J=big)
    assert rc == 1 and "sum of |J|" in msg
    rc, msg = _create(P, betas=np.array([1.0, 2.0, 0.5]))
    assert rc == 1 and "descending" in msg
    assert _create(P, betas=np.array([1.0, 0.0]))[0] == 1
    assert _create(P, nt=65, betas=W.beta_ladder(65, 0.1, 3.0))[0] == 1
    assert _create(P, R=0)[0] == 1
    assert _create(P, R=1025)[0] == 1
    # a beta gap so small that the exchange table would exceed 2^22 entries
    rc, msg = _create(P, betas=np.array([1.0, 1.0 - 1e-9]))
    assert rc == 1 and "2^22" in msg


def test_int_issue_microbenchmark_validates_arguments(P):
    C = ctypes
    lib = P.load()
    ops, ms = C.c_double(), C.c_double()
    for kind, iters, reps in [(-1, 16, 1), (5, 16, 1), (0, 0, 1), (0, (1 << 22) + 1, 1), (0, 16, 0),
                              (0, 16, 1001)]:
        assert lib.pt_int_issue_rate(kind, iters, reps, C.byref(ops), C.byref(ms), None) == 1
    assert lib.pt_int_issue_rate(0, 16, 1, None, C.byref(ms), None) == 1
    assert "ops_per_s" in lib.pt_last_error(None).decode()
    with pytest.raises(ValueError):
        P.int_issue_rate("fp32")


def test_python_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_1605_03607_gb300._lib as lib
    monkeypatch.setattr(lib, "_lib", None)
    monkeypatch.setattr(lib, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        lib.load()


def test_graph_form_validation_without_gpu(P):
    """pt_create_graph rejects coupler lists that are not sets of C_L couplers
    (checked on the host before any device work)."""
    lib = P.load()
    L = 2
    import oracle
    ei, ej = oracle.chimera_edges(L)
    betas = W.beta_ladder(4, 0.5, 3.0)

    def create(a, b, n=8 * L * L):
        a = np.ascontiguousarray(a, np.int32)
        b = np.ascontiguousarray(b, np.int32)
        J = np.ones(len(a), np.int8)
        g = P._lib.pt_graph(n, len(a), a.ctypes.data, b.ctypes.data, L)
        h = ctypes.c_void_p()
        rc = lib.pt_create_graph(ctypes.byref(h), ctypes.byref(g), J.ctypes.data_as(ctypes.c_void_p),
                                 betas.ctypes.data_as(ctypes.c_void_p), len(betas), 2, 1, 0, None)
        return rc, lib.pt_last_error(None).decode()

    rc, msg = create([0, 0], [1, 2])                  # spins 0-1, 0-2: same orientation in one cell
    assert rc == 1 and "not an edge" in msg
    rc, msg = create([0, 4], [4, 0])                  # the same coupler in both orientations
    assert rc == 1 and "twice" in msg
    rc, msg = create([0], [8])                        # vertical k=0 of cell (0,0) to horizontal cell (0,1): no
    assert rc == 1 and "not an edge" in msg
    rc, msg = create(ei[:3], ej[:3], n=31)
    assert rc == 1 and "8 L^2" in msg
