"""GPU surrogate (BF16 tensor-core forward/backward, FP32 Adam) vs the FP64 oracle.

Tolerances: predictions and gradients within 2e-2 relative of the FP64
forward/backward (BF16 weights and activations, FP32 accumulation); the Adam
update, which is FP32 elementwise arithmetic on the GPU's own gradient,
within 1e-5.
"""
import numpy as np
import pytest

import workloads as W
from oracle import surrogate as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1605_03607_gb300 as pkg
    from paper_1605_03607_gb300 import build as b
    b.build()
    pkg.load()
    return pkg


def _J(L, B, seed):
    return np.random.default_rng(seed).choice([-3, -2, -1, 1, 2, 3], size=(B, W.chimera_n_edges(L))).astype(np.int8)


def _theta(seed):
    rng = np.random.default_rng(seed)
    th = W.surrogate_init_params(seed)
    return th + 0.02 * rng.standard_normal(len(th))


def _rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-12)


@pytest.mark.parametrize("L,B", [(1, 5), (2, 3), (4, 4), (8, 2)])
def test_forward_matches_fp64(P, L, B):
    th = _theta(L)
    J = _J(L, B, 10 + L)
    with P.Surrogate() as m:
        m.set_params(th)
        y = m.forward(L, J)
    ref = S.forward(th.astype(np.float32).astype(np.float64), L, J)
    assert np.all(np.abs(y - ref) <= 2e-2 * np.maximum(np.abs(ref), 1.0)), (y, ref)


@pytest.mark.parametrize("L,B", [(1, 4), (2, 3), (4, 2)])
def test_gradient_matches_bf16_storage_model(P, L, B):
    """Against the oracle's BF16-storage model the GPU gradient is tight on
    every size, including one K_{4,4} cell, where BF16 rounding flips enough
    ReLU masks to move the gradient ~8 % away from exact FP64."""
    th = _theta(20 + L)
    J = _J(L, B, 30 + L)
    t = np.random.default_rng(L).uniform(1.5, 4.0, B)
    with P.Surrogate() as m:
        m.set_params(th)
        loss, g = m.grad(L, J, t)
    th64 = th.astype(np.float32).astype(np.float64)
    _, rg = S.loss_and_grad(th64, L, J, t, bf16=True)
    assert _rel(g, rg) <= 5e-3, _rel(g, rg)


@pytest.mark.parametrize("L,B", [(2, 3), (4, 2), (8, 2)])
def test_gradient_matches_fp64(P, L, B):
    th = _theta(20 + L)
    J = _J(L, B, 30 + L)
    t = np.random.default_rng(L).uniform(1.5, 4.0, B)
    with P.Surrogate() as m:
        m.set_params(th)
        loss, g = m.grad(L, J, t)
    th64 = th.astype(np.float32).astype(np.float64)
    rloss, rg = S.loss_and_grad(th64, L, J, t)
    assert abs(loss - rloss) <= 2e-2 * max(abs(rloss), 1e-6)
    assert _rel(g, rg) <= 2e-2, _rel(g, rg)
    # every parameter tensor on its own, where its reference gradient is not negligible
    o = 0
    for name, n, _ in W.surrogate_param_sizes():
        seg, rseg = g[o:o + n], rg[o:o + n]
        if np.linalg.norm(rseg) > 1e-3 * np.linalg.norm(rg):
            assert _rel(seg, rseg) <= 5e-2, (name, _rel(seg, rseg))
        o += n


def test_adam_step_matches_fp64(P):
    th = _theta(7)
    J = _J(2, 3, 7)
    t = np.array([2.0, 3.0, 2.5])
    with P.Surrogate() as m:
        m.set_params(th)
        _, g1 = m.grad(2, J, t)
        m.adam(1e-3)
        th1 = m.params()
        _, g2 = m.grad(2, J, t)
        m.adam(1e-3)
        th2 = m.params()
    th32 = th.astype(np.float32).astype(np.float64)
    r1, mo, ve = S.adam_step(th32, g1.astype(np.float64), np.zeros(len(th)), np.zeros(len(th)), 1)
    assert np.allclose(th1, r1, rtol=1e-5, atol=1e-6)
    r2, _, _ = S.adam_step(th1.astype(np.float64), g2.astype(np.float64), mo, ve, 2)
    assert np.allclose(th2, r2, rtol=1e-5, atol=1e-6)


def test_training_reduces_loss(P):
    L, B = 4, 32
    J = _J(L, B, 3)
    rng = np.random.default_rng(3)
    t = 2.0 + 0.5 * (J == 3).mean(axis=1) * 10 + 0.01 * rng.standard_normal(B)   # a learnable target
    with P.Surrogate() as m:
        m.set_params(W.surrogate_init_params(1))
        first = m.train_step(L, J, t, 1e-3)
        for _ in range(150):
            last = m.train_step(L, J, t, 1e-3)
    assert last < 0.2 * first, (first, last)


def test_rejects_zero_couplers(P):
    J = _J(2, 1, 1)
    J[0, 3] = 0
    with P.Surrogate() as m:
        with pytest.raises(P.PTError):
            m.forward(2, J)
