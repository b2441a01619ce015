"""FP64 oracle of the surrogate network (TEST INFRASTRUCTURE ONLY).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may use
this module.  Plain NumPy float64, written from the network definition below;
it shares nothing with the CUDA kernels.

The surrogate predicts log10 TTS of a Chimera instance (the hardness figure of
merit of Sec. II) from its couplers, so that the RAO loop (Algorithm 1) only
spends PT evaluations on promising proposals.  The paper has no surrogate;
the architecture is this library's:

  inputs   h0_i = X[u_i]            (u_i: orientation of spin i, 2 rows)
           e0_e = Jt[idx(J_e)]      (idx: -3,-2,-1,1,2,3 -> 0..5)
  layer l  m_i  = sum_{j in N(i)} relu(Wm [h_j , e_ij] + bm)
           h_i <- h_i + relu(Wu [h_i , m_i] + bu)
           e_ij <- e_ij + relu(We [e_ij , h_i + h_j] + be)      (new h)
  readout  g = mean_i h_i ; a = relu(W1 g + b1) ; y = w2 . a + b2
  loss     mean over the batch of (y - t)^2

Parameters are one flat vector (the interface shared with the GPU library):
  X[2,H], Jt[6,H], per layer (Wm[H,2H], bm[H], Wu[H,2H], bu[H], We[H,2H], be[H]),
  W1[H,H], b1[H], w2[H], b2[1]   (matrices row-major, rows = outputs).
"""
from __future__ import annotations

import numpy as np

J_INDEX = {-3: 0, -2: 1, -1: 2, 1: 3, 2: 4, 3: 5}


def param_shapes(H=64, layers=4):
    shapes = [("X", (2, H)), ("Jt", (6, H))]
    for l in range(layers):
        shapes += [(f"Wm{l}", (H, 2 * H)), (f"bm{l}", (H,)), (f"Wu{l}", (H, 2 * H)), (f"bu{l}", (H,)),
                   (f"We{l}", (H, 2 * H)), (f"be{l}", (H,))]
    shapes += [("W1", (H, H)), ("b1", (H,)), ("w2", (H,)), ("b2", (1,))]
    return shapes


def n_params(H=64, layers=4):
    return int(sum(np.prod(s) for _, s in param_shapes(H, layers)))


def unpack(theta, H=64, layers=4):
    out, o = {}, 0
    for name, s in param_shapes(H, layers):
        n = int(np.prod(s))
        out[name] = np.asarray(theta[o:o + n], np.float64).reshape(s)
        o += n
    assert o == len(theta)
    return out


def pack(p, H=64, layers=4):
    return np.concatenate([np.asarray(p[name], np.float64).ravel() for name, _ in param_shapes(H, layers)])


def chimera_graph(L):
    """Edges (ei, ej) in the library's coupler order and each spin's orientation."""
    ei, ej = [], []
    idx = lambda r, c, u, k: 8 * (r * L + c) + 4 * u + k
    for r in range(L):
        for c in range(L):
            for k in range(4):
                for kp in range(4):
                    ei.append(idx(r, c, 0, k)); ej.append(idx(r, c, 1, kp))
    for r in range(L - 1):
        for c in range(L):
            for k in range(4):
                ei.append(idx(r, c, 0, k)); ej.append(idx(r + 1, c, 0, k))
    for r in range(L):
        for c in range(L - 1):
            for k in range(4):
                ei.append(idx(r, c, 1, k)); ej.append(idx(r, c + 1, 1, k))
    u = np.array([(i >> 2) & 1 for i in range(8 * L * L)])
    return np.array(ei), np.array(ej), u


def relu(x):
    return np.maximum(x, 0.0)


def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even) and return float64."""
    a = np.ascontiguousarray(x, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _identity(x):
    return x


# bf16=True models a BF16-storage implementation: the per-layer weight
# matrices, the embedded inputs, every stored activation (m, updated h, s,
# updated e) and every backward pre-activation gradient dZ are rounded to
# bfloat16, while all sums stay in float64.  It is a precision model used to
# separate rounding from mistakes on graphs too small for the 2e-2 bar; the
# default (bf16=False) is the exact float64 network.
def forward(theta, L, J, H=64, layers=4, keep=False, bf16=False):
    """J: [B, E] couplers.  Returns y [B] (and the saved activations if keep)."""
    q = bf16_round if bf16 else _identity
    p = unpack(theta, H, layers)
    ei, ej, u = chimera_graph(L)
    J = np.atleast_2d(np.asarray(J))
    B, N = J.shape[0], 8 * L * L
    jidx = np.vectorize(J_INDEX.__getitem__)(J)
    h = q(np.repeat(p["X"][u][None], B, axis=0))                   # [B, N, H]
    e = q(p["Jt"][jidx])                                           # [B, E, H]
    saved = []
    for l in range(layers):
        Wm, bm, Wu, bu, We, be = (p[f"{n}{l}"] for n in ("Wm", "bm", "Wu", "bu", "We", "be"))
        Wm, Wu, We = q(Wm), q(Wu), q(We)
        # messages in both directions of every edge
        zf = np.concatenate([h[:, ej], e], -1) @ Wm.T + bm          # j -> i  (to ei)
        zb = np.concatenate([h[:, ei], e], -1) @ Wm.T + bm          # i -> j  (to ej)
        m = np.zeros_like(h)
        for b in range(B):
            np.add.at(m[b], ei, relu(zf[b]))
            np.add.at(m[b], ej, relu(zb[b]))
        m = q(m)
        zu = np.concatenate([h, m], -1) @ Wu.T + bu
        h2 = q(h + relu(zu))
        s = q(h2[:, ei] + h2[:, ej])
        ze = np.concatenate([e, s], -1) @ We.T + be
        e2 = q(e + relu(ze))
        saved.append((h, e, zf, zb, m, zu, h2, s, ze))
        h, e = h2, e2
    g = h.mean(axis=1)                                             # [B, H]
    z1 = g @ p["W1"].T + p["b1"]
    a = relu(z1)
    y = a @ p["w2"] + p["b2"][0]
    if keep:
        return y, dict(saved=saved, g=g, z1=z1, a=a, h=h, e=e, jidx=jidx, u=u, ei=ei, ej=ej)
    return y


def loss_and_grad(theta, L, J, t, H=64, layers=4, bf16=False):
    """MSE loss mean_b (y_b - t_b)^2 and its gradient with respect to theta."""
    q = bf16_round if bf16 else _identity
    p = unpack(theta, H, layers)
    y, c = forward(theta, L, J, H, layers, keep=True, bf16=bf16)
    t = np.asarray(t, np.float64)
    B = y.shape[0]
    N = 8 * L * L
    ei, ej, u, jidx = c["ei"], c["ej"], c["u"], c["jidx"]
    loss = np.mean((y - t) ** 2)
    g = {k: np.zeros_like(v) for k, v in p.items()}
    dy = 2.0 * (y - t) / B                                         # [B]
    g["w2"] = c["a"].T @ dy
    g["b2"] = np.array([dy.sum()])
    da = dy[:, None] * p["w2"][None]
    dz1 = da * (c["z1"] > 0)
    g["W1"] = dz1.T @ c["g"]
    g["b1"] = dz1.sum(0)
    dg = dz1 @ p["W1"]                                             # [B, H]
    dh = np.repeat(dg[:, None, :] / N, N, axis=1)                  # grad wrt final h
    de = np.zeros_like(c["e"])                                     # grad wrt final e (unused by readout)
    for l in reversed(range(layers)):
        h, e, zf, zb, m, zu, h2, s, ze = c["saved"][l]
        Wm, Wu, We = q(p[f"Wm{l}"]), q(p[f"Wu{l}"]), q(p[f"We{l}"])
        # edge update e2 = e + relu(ze), ze = We [e, s] + be, s = h2_i + h2_j
        dze = q(de * (ze > 0))
        g[f"We{l}"] = np.einsum("beo,bei->oi", dze, np.concatenate([e, s], -1))
        g[f"be{l}"] = dze.sum((0, 1))
        dx = dze @ We                                              # [B, E, 2H]
        de_in = de + dx[..., :H]
        ds = dx[..., H:]
        dh2 = dh.copy()
        for b in range(B):
            np.add.at(dh2[b], ei, ds[b])
            np.add.at(dh2[b], ej, ds[b])
        # node update h2 = h + relu(zu), zu = Wu [h, m] + bu
        dzu = q(dh2 * (zu > 0))
        g[f"Wu{l}"] = np.einsum("bno,bni->oi", dzu, np.concatenate([h, m], -1))
        g[f"bu{l}"] = dzu.sum((0, 1))
        dxu = dzu @ Wu
        dh_in = dh2 + dxu[..., :H]
        dm = dxu[..., H:]
        # messages m_i = sum relu(zf) (to ei) + relu(zb) (to ej)
        dzf = q(dm[:, ei] * (zf > 0))
        dzb = q(dm[:, ej] * (zb > 0))
        g[f"Wm{l}"] = (np.einsum("beo,bei->oi", dzf, np.concatenate([h[:, ej], e], -1)) +
                       np.einsum("beo,bei->oi", dzb, np.concatenate([h[:, ei], e], -1)))
        g[f"bm{l}"] = dzf.sum((0, 1)) + dzb.sum((0, 1))
        dxf = dzf @ Wm
        dxb = dzb @ Wm
        for b in range(B):
            np.add.at(dh_in[b], ej, dxf[b][:, :H])
            np.add.at(dh_in[b], ei, dxb[b][:, :H])
        de_in = de_in + dxf[..., H:] + dxb[..., H:]
        dh, de = dh_in, de_in
    for b in range(B):
        np.add.at(g["X"], u, dh[b])
        np.add.at(g["Jt"], jidx[b], de[b])
    return loss, pack(g, H, layers)


def adam_step(theta, grad, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) with bias correction; step counts from 1."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
