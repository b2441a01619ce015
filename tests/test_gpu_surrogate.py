"""GPU surrogate (BF16 tensor-core forward/backward, FP32 Adam) vs the FP64 oracle.

The reference point.  The network trains with FP32 master weights and
multiplies with their BF16 copies (the three per-layer matrices Wm, Wu, We);
the gradient it produces is the gradient at those BF16 values, which is what
mixed-precision training applies to the masters.  The FP64 oracle is
therefore evaluated at the same parameter point: the per-layer matrices
rounded to BF16, every other parameter (embeddings, biases, readout) as the
FP32 value the kernels read.  Only the parameters are rounded; the oracle's
arithmetic is plain FP64.

Tolerances (stated once, used below):
  * predictions: |y - y_ref| <= 2e-2 max(|y_ref|, 1), element by element;
  * loss: within 2e-2 relative;
  * gradient, every parameter tensor T on its own:
      ||g_T - ref_T|| <= 2e-2 ||ref_T||                       (relative L2)
      |g_i - ref_i| <= 2e-2 max(|ref_i|, FLOOR * max|ref_T|)  (element-wise)
    with FLOOR = 2.  The floor is there because the batch-summed gradient
    of a bias or of the readout cancels: with BF16 activations each
    graph's prediction carries an error of a few 1e-4, and where
    sum_b (y_b - t_b) is small the relative error of the sum grows without
    bound while its absolute error stays at the per-graph level.  Every
    element larger than 2 % of its tensor's largest must still have the
    right sign and be within 4 % of that largest element.
  * Adam: FP32 elementwise arithmetic on the GPU's own gradient, 1e-5.

Sizes reach the full training batch (256 C_8 graphs: 753,664 message rows,
about 39 row chunks per persistent weight-gradient CTA) and a batch of single
K_{4,4} cells.  One cell with a batch of 4 (64 message rows) is not checked
here: there a single ReLU mask that flips between the BF16 and FP64 forward
moves a whole tensor's gradient by several percent.
"""
import numpy as np
import pytest

import workloads as W
from oracle import surrogate as S

pytestmark = pytest.mark.gpu

FLOOR = 2.0


@pytest.fixture(scope="module")
def P():
    import paper_1605_03607_gb300 as pkg
    from paper_1605_03607_gb300 import build as b
    b.build()
    pkg.load()
    return pkg


def _J(L, B, rng):
    return rng.choice([-3, -2, -1, 1, 2, 3], size=(B, W.chimera_n_edges(L))).astype(np.int8)


def _theta(seed, rng):
    th = W.surrogate_init_params(seed)
    return (th + 0.02 * rng.standard_normal(len(th))).astype(np.float32)


def _at_bf16_layer_weights(theta32):
    """The parameter point the kernels compute with: per-layer matrices in
    BF16, everything else the FP32 value."""
    th = theta32.astype(np.float64)
    o = 0
    for name, n, _ in W.surrogate_param_sizes():
        if name[0] == "W" and name[1] in "mue":
            th[o:o + n] = S.bf16_round(th[o:o + n])
        o += n
    return th


@pytest.mark.parametrize("L,B", [(1, 5), (2, 3), (4, 4), (8, 2), (8, 256)])
def test_forward_matches_fp64(P, L, B):
    rng = np.random.default_rng(100 + L + B)
    th = _theta(L, rng)
    J = _J(L, B, rng)
    with P.Surrogate() as m:
        m.set_params(th)
        y = m.forward(L, J)
    for ref in (S.forward(th.astype(np.float64), L, J), S.forward(_at_bf16_layer_weights(th), L, J)):
        assert np.all(np.abs(y - ref) <= 2e-2 * np.maximum(np.abs(ref), 1.0)), (y, ref)


@pytest.mark.parametrize("L,B", [(1, 256), (2, 64), (4, 64), (8, 2), (8, 256)])
def test_gradient_matches_fp64_per_tensor_and_element(P, L, B):
    rng = np.random.default_rng(200 + L + B)
    th = _theta(20 + L, rng)
    J = _J(L, B, rng)
    t = rng.uniform(1.5, 4.0, B)
    with P.Surrogate() as m:
        m.set_params(th)
        loss, g = m.grad(L, J, t)
    rloss, rg = S.loss_and_grad(_at_bf16_layer_weights(th), L, J, t)
    assert abs(loss - rloss) <= 2e-2 * max(abs(rloss), 1e-6)
    o, checked = 0, 0
    for name, n, _ in W.surrogate_param_sizes():
        a, b = g[o:o + n].astype(np.float64), rg[o:o + n]
        o += n
        top = np.abs(b).max()
        if top == 0.0:                      # the last layer's edge update does not reach the readout
            assert np.all(a == 0.0), name
            continue
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert rel <= 2e-2, (name, rel)
        bad = np.abs(a - b) > 2e-2 * np.maximum(np.abs(b), FLOOR * top)
        assert not bad.any(), (name, int(bad.sum()), float(np.abs(a - b).max() / top))
        checked += 1
    assert checked >= 26


def test_adam_step_matches_fp64(P):
    rng = np.random.default_rng(7)
    th = _theta(7, rng)
    J = _J(2, 3, rng)
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
    rng = np.random.default_rng(3)
    J = _J(L, B, rng)
    t = 2.0 + 0.5 * (J == 3).mean(axis=1) * 10 + 0.01 * rng.standard_normal(B)   # a learnable target
    with P.Surrogate() as m:
        m.set_params(W.surrogate_init_params(1))
        first = m.train_step(L, J, t, 1e-3)
        for _ in range(150):
            last = m.train_step(L, J, t, 1e-3)
    assert last < 0.2 * first, (first, last)


def test_training_is_bit_reproducible(P):
    """Every reduction of a training step runs in a fixed order (no floating-point
    atomics), so two models trained from the same parameters on the same batches
    end bit-identical, at a batch large enough for many CTAs per kernel."""
    L, B = 4, 96
    rng = np.random.default_rng(5)
    batches = [(_J(L, B, rng), 2.0 + 0.3 * rng.standard_normal(B)) for _ in range(3)]
    thetas, losses = [], []
    for _ in range(2):
        with P.Surrogate() as m:
            m.set_params(W.surrogate_init_params(1))
            losses.append([m.train_step(L, J, t, 1e-3) for J, t in batches * 2])
            thetas.append(m.params())
    assert losses[0] == losses[1]
    assert np.array_equal(thetas[0], thetas[1])


def test_rejects_zero_couplers(P):
    J = _J(2, 1, np.random.default_rng(1))
    J[0, 3] = 0
    with P.Surrogate() as m:
        with pytest.raises(P.PTError):
            m.forward(2, J)
