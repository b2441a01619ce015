"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and bench.py.

This module holds no part of the method's arithmetic: no energies, no Monte Carlo,
no random-number stream the method itself draws.  It only produces the inputs a
caller hands to either implementation:

* the size of an ideal Chimera graph C_L (L x L unit cells of K_{4,4}, 8 spins
  per cell; the graph of Appendix A / Fig. 8, all qubits present);
* a random coupler vector J with values uniform on {-3,-2,-1,1,2,3}
  (the paper's instances are J = +-1, Algorithm 1; the wider range is the
  workload this library is measured on, with zero fields as in Eq. 1);
* a geometric inverse-temperature ladder (the paper's PT uses a fixed grid of
  N_T temperatures T_1 < ... < T_NT, Sec. II; slot 0 is the coldest here);
* the named workload configurations.

Everything is deterministic in (seed, uid).
"""
from __future__ import annotations

import numpy as np

J_VALUES = np.array([-3, -2, -1, 1, 2, 3], dtype=np.int8)


def chimera_n_spins(L: int) -> int:
    """Number of spins of the ideal Chimera graph C_L (8 per unit cell)."""
    return 8 * L * L


def chimera_n_edges(L: int) -> int:
    """Number of couplers of C_L: 16 per cell plus 4 per adjacent cell pair."""
    return 16 * L * L + 8 * L * (L - 1)


def random_couplers(L: int, seed: int, uid: int) -> np.ndarray:
    """J_e uniform on {-3,-2,-1,1,2,3} for every coupler of C_L, keyed by (seed, uid)."""
    rng = np.random.Generator(np.random.Philox(key=[seed & 0xFFFFFFFF, uid & 0xFFFFFFFF]))
    idx = rng.integers(0, 6, size=chimera_n_edges(L))
    return J_VALUES[idx].copy()


def random_pm1_couplers(L: int, seed: int, uid: int) -> np.ndarray:
    """J_e uniform on {-1,+1} (the paper's signed instances, Algorithm 1)."""
    rng = np.random.Generator(np.random.Philox(key=[seed & 0xFFFFFFFF, uid & 0xFFFFFFFF]))
    return np.where(rng.integers(0, 2, size=chimera_n_edges(L)) == 0, -1, 1).astype(np.int8)


def beta_ladder(n_temps: int, beta_min: float, beta_max: float) -> np.ndarray:
    """Geometric ladder, strictly descending: slot 0 is the coldest (beta_max)."""
    if n_temps == 1:
        return np.array([beta_max], dtype=np.float64)
    t = np.arange(n_temps, dtype=np.float64)
    return beta_max * np.power(beta_min / beta_max, t / (n_temps - 1))


def random_spins(shape, seed: int) -> np.ndarray:
    """+-1 int8 spins (used for caller-supplied initial states in tests)."""
    rng = np.random.default_rng(seed)
    return np.where(rng.integers(0, 2, size=shape) == 0, -1, 1).astype(np.int8)


# Named workloads.  Seeds follow seed = 20160511 + index; uid = instance index.
CONFIGS = {
    # Tiny plain case: C_4, 16 temperatures in [0.1, 3], 8 runs x 2048 sweeps,
    # exchange every sweep, target = best energy of the same pass, 20 RAO steps.
    "c4_tiny": dict(L=4, n_temps=16, beta_min=0.1, beta_max=3.0, n_runs=8,
                    sweeps=2048, pass_mult=1, exchange_every=1, steps=20,
                    seed=20160511),
    # One C_8 instance: 32 temperatures in [0.1, 4], 64 runs, TTS horizon 2^16
    # sweeps, target = best energy of a 4x longer pass, 200 RAO steps.
    "c8_single": dict(L=8, n_temps=32, beta_min=0.1, beta_max=4.0, n_runs=64,
                      sweeps=1 << 16, pass_mult=4, exchange_every=1, steps=200,
                      seed=20160512),
    # Batched: 256 instances mixed evenly over C_4/C_8/C_12/C_16, 24..48
    # temperatures (uneven), 32 runs each, 2^14 sweeps.
    "batched_256": dict(n_instances=256, Ls=(4, 8, 12, 16), n_runs=32,
                        sweeps=1 << 14, beta_min=0.1, beta_max=4.0,
                        exchange_every=1, seed=20160513),
    # Surrogate-guided engineering at C_16: 48 temperatures in [0.05, 5], 32 runs.
    "c16_guided": dict(L=16, n_temps=48, beta_min=0.05, beta_max=5.0, n_runs=32,
                       sweeps=1 << 12, max_sweeps=1 << 20, exchange_every=1,
                       proposals=64, top=4, seed=20160515),
}


def surrogate_param_sizes(H=64, layers=4):
    """Sizes of the surrogate's flat parameter vector, in order: embeddings
    X[2,H], Jt[6,H]; per layer Wm[H,2H], bm[H], Wu[H,2H], bu[H], We[H,2H], be[H];
    readout W1[H,H], b1[H], w2[H], b2[1]."""
    sizes = [("X", 2 * H, 2), ("Jt", 6 * H, 6)]
    for l in range(layers):
        for n in ("m", "u", "e"):
            sizes += [(f"W{n}{l}", 2 * H * H, 2 * H), (f"b{n}{l}", H, 0)]
    sizes += [("W1", H * H, H), ("b1", H, 0), ("w2", H, H), ("b2", 1, 0)]
    return sizes


def surrogate_init_params(seed, H=64, layers=4):
    """Initial surrogate parameters: weights uniform in +-1/sqrt(fan_in),
    embeddings uniform in +-1, biases 0 except the output bias (3, a typical
    log10 TTS)."""
    rng = np.random.default_rng(seed)
    out = []
    for name, n, fan_in in surrogate_param_sizes(H, layers):
        if name in ("X", "Jt"):
            out.append(rng.uniform(-1, 1, n))
        elif fan_in > 0:
            out.append(rng.uniform(-1, 1, n) / np.sqrt(fan_in))
        elif name == "b2":
            out.append(np.array([3.0]))
        else:
            out.append(np.zeros(n))
    return np.concatenate(out)


def batched_instances(cfg=None):
    """Instance list of the batched workload: (L, n_temps, J, betas, uid)."""
    cfg = cfg or CONFIGS["batched_256"]
    out = []
    n = cfg["n_instances"]
    Ls = cfg["Ls"]
    for i in range(n):
        L = Ls[i * len(Ls) // n]
        nt = 24 + (7 * i) % 25
        J = random_couplers(L, cfg["seed"], i)
        betas = beta_ladder(nt, cfg["beta_min"], cfg["beta_max"])
        out.append(dict(L=L, n_temps=nt, J=J, betas=betas, uid=i))
    return out
