"""Pins of the FP64 surrogate oracle (no GPU).

Finite differences pin the backward pass to the forward pass; closed forms,
symmetries of the Chimera graph and the Adam update pin the forward pass and
the optimiser themselves.
"""
import numpy as np
import pytest

import workloads as W
from oracle import surrogate as S


def _rand_J(L, B, seed):
    return np.random.default_rng(seed).choice([-3, -2, -1, 1, 2, 3], size=(B, W.chimera_n_edges(L)))


def test_layout_matches_inputs_module():
    for H, layers in ((64, 4), (8, 2)):
        assert S.n_params(H, layers) == sum(n for _, n, _ in W.surrogate_param_sizes(H, layers))
        assert [n for n, _ in S.param_shapes(H, layers)] == [n for n, _, _ in W.surrogate_param_sizes(H, layers)]
    assert S.n_params() == len(W.surrogate_init_params(0))


def test_graph_matches_chimera():
    import oracle
    for L in (1, 2, 4):
        ei, ej, u = S.chimera_graph(L)
        oi, oj = oracle.chimera_edges(L)
        assert np.array_equal(ei, oi) and np.array_equal(ej, oj)


@pytest.mark.parametrize("H,layers,L,B", [(6, 2, 1, 3), (8, 2, 2, 2)])
def test_gradient_matches_central_differences(H, layers, L, B):
    rng = np.random.default_rng(5)
    theta = W.surrogate_init_params(3, H, layers) + 0.05 * rng.standard_normal(S.n_params(H, layers))
    J = _rand_J(L, B, 7)
    t = rng.uniform(1, 4, B)
    loss, g = S.loss_and_grad(theta, L, J, t, H, layers)
    idx = rng.choice(len(theta), size=min(len(theta), 120), replace=False)
    eps = 1e-6
    for k in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[k] += eps
        tm[k] -= eps
        fd = (np.mean((S.forward(tp, L, J, H, layers) - t) ** 2) -
              np.mean((S.forward(tm, L, J, H, layers) - t) ** 2)) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-3 * max(abs(fd), abs(g[k])) + 1e-7, (k, fd, g[k])


def test_gradient_full_size_sampled():
    rng = np.random.default_rng(11)
    theta = W.surrogate_init_params(4)
    J = _rand_J(2, 2, 3)
    t = np.array([2.0, 3.5])
    loss, g = S.loss_and_grad(theta, 2, J, t)
    eps = 1e-6
    for k in rng.choice(len(theta), size=40, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[k] += eps
        tm[k] -= eps
        fd = (np.mean((S.forward(tp, 2, J) - t) ** 2) - np.mean((S.forward(tm, 2, J) - t) ** 2)) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-3 * max(abs(fd), abs(g[k])) + 1e-7


def test_readout_bias_only():
    H, layers = 8, 2
    theta = np.zeros(S.n_params(H, layers))
    theta[-1] = 2.75
    assert np.allclose(S.forward(theta, 2, _rand_J(2, 3, 1), H, layers), 2.75)


def test_message_sum_closed_form():
    """Zero weights, message bias c: every node receives deg(i) * c per channel,
    so with Wu = [0 | I] and W1 = I, w2 = 1/H the output is c * 2E / N."""
    H, layers, c = 4, 1, 0.3
    p = S.unpack(np.zeros(S.n_params(H, layers)), H, layers)
    p["bm0"][:] = c
    p["Wu0"][:, H:] = np.eye(H)
    p["W1"][:] = np.eye(H)
    p["w2"][:] = 1.0 / H
    theta = S.pack(p, H, layers)
    for L in (1, 2, 3):
        E, N = W.chimera_n_edges(L), 8 * L * L
        y = S.forward(theta, L, _rand_J(L, 2, L), H, layers)
        assert np.allclose(y, c * 2 * E / N)


def test_chimera_automorphisms_leave_prediction_unchanged():
    """Relabelling k inside every cell, or mirroring the grid, is a graph
    automorphism that keeps orientations: the prediction must not change."""
    L, H, layers = 3, 8, 2
    theta = W.surrogate_init_params(9, H, layers)
    J = _rand_J(L, 1, 4)[0]
    ei, ej, u = S.chimera_graph(L)
    key = {(min(a, b), max(a, b)): e for e, (a, b) in enumerate(zip(ei, ej))}

    def relabel(f):
        J2 = np.zeros_like(J)
        for e, (a, b) in enumerate(zip(ei, ej)):
            fa, fb = f(a), f(b)
            J2[key[(min(fa, fb), max(fa, fb))]] = J[e]
        return J2

    def coords(i):
        cell, rem = divmod(i, 8)
        r, c = divmod(cell, L)
        return r, c, rem // 4, rem % 4

    perm = [2, 0, 3, 1]
    f_k = lambda i: (lambda r, c, uu, k: 8 * (r * L + c) + 4 * uu + perm[k])(*coords(i))
    f_row = lambda i: (lambda r, c, uu, k: 8 * ((L - 1 - r) * L + c) + 4 * uu + k)(*coords(i))
    y0 = S.forward(theta, L, J[None], H, layers)
    for f in (f_k, f_row):
        assert np.allclose(S.forward(theta, L, relabel(f)[None], H, layers), y0, rtol=1e-12)
    # a map that is not an automorphism of the coupler values (one coupler changed) does change it
    J3 = J.copy()
    J3[0] = -J3[0]
    assert not np.allclose(S.forward(theta, L, J3[None], H, layers), y0)


def test_bf16_rounding_matches_library():
    torch = pytest.importorskip("torch")
    x = np.concatenate([np.random.default_rng(0).standard_normal(10000) * 10.0 ** np.arange(-5, 5).repeat(1000),
                        [1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, -0.0, 3.0e38]])
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(S.bf16_round(x), want)
    assert S.bf16_round(np.array([1.0 + 2.0 ** -8]))[0] == 1.0          # tie goes to even


def test_bf16_model_close_to_fp64_on_workload_sizes():
    theta = W.surrogate_init_params(2)
    J = _rand_J(4, 2, 5)
    t = np.array([2.0, 3.0])
    _, g = S.loss_and_grad(theta, 4, J, t)
    _, gq = S.loss_and_grad(theta, 4, J, t, bf16=True)
    assert np.linalg.norm(gq - g) / np.linalg.norm(g) < 2e-2


def test_adam_first_step_closed_form():
    theta = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    t2, m, v = S.adam_step(theta, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    # first step: m_hat = g, v_hat = g^2, update = lr * g / (|g| + eps)
    assert np.allclose(t2, theta - 0.01 * g / (np.abs(g) + 1e-8))
    t3, _, _ = S.adam_step(t2, g, m, v, 2, lr=0.01)
    assert np.allclose(t3, t2 - 0.01 * g / (np.abs(g) + 1e-8))     # constant gradient keeps the step
