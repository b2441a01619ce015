"""The kernels' split forms of Philox4x32-10, run on the host (no GPU needed).

`csrc/pt_philox.cuh` is host-and-device code. The sweeps draw their
Metropolis uniforms from counter (s, run << 16 | slot, group, 0):
  * the slot-major mapping through philox_sweep_pre + philox_group_prod,
    with round 0's product of the group index kept per cell;
  * the cell-major mapping through philox_pre + philox_slot;
  * the exchange preparation and the initial state through philox10.
This test compiles the header with the host compiler. On seeded counters of
that form it checks two things:
  * every split form equals the plain generator;
  * the plain generator equals the oracle's, which is itself pinned to the
    published known-answer vectors.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

HEADER = os.path.join(os.path.dirname(__file__), "..", "paper_1605_03607_gb300", "csrc", "pt_philox.cuh")

DRIVER = r"""
#define __host__
#define __device__
#define __forceinline__ inline
#include <cstdint>
#include <cstdio>
struct uint4 { uint32_t x, y, z, w; };
static inline uint4 make_uint4(uint32_t a, uint32_t b, uint32_t c, uint32_t d) { return {a, b, c, d}; }
#include "pt_philox.cuh"
using namespace ptg;
int main() {
    unsigned s, c1, g, k0, k1;
    while (std::scanf("%u %u %u %u %u", &s, &c1, &g, &k0, &k1) == 5) {
        const uint4 a = philox10(s, c1, g, 0u, k0, k1);
        const uint64_t B = (uint64_t)PHILOX_M1 * g;
        const uint4 b = philox_group_prod(philox_sweep_pre(s, k0, k1), c1, (uint32_t)(B >> 32), (uint32_t)B, k0, k1);
        const uint4 c = philox_slot(philox_pre(s, g, k0, k1), c1, k0, k1);
        std::printf("%u %u %u %u %u %u %u %u %u %u %u %u\n", a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w,
                    c.x, c.y, c.z, c.w);
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("philox")
    src = d / "split.cpp"
    src.write_text(DRIVER)
    exe = d / "split"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.dirname(os.path.abspath(HEADER)), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    return str(exe)


def test_split_forms_equal_plain_generator_and_oracle(driver):
    rng = np.random.default_rng(1605)
    n = 4096
    s = rng.integers(0, 2**32, n, dtype=np.uint64)
    s[:256] = np.arange(256)                                          # small sweep counts
    run = rng.integers(0, 1 << 16, n, dtype=np.uint64)
    slot = rng.integers(0, 64, n, dtype=np.uint64)
    c1 = (run << 16) | slot
    g = rng.integers(0, 2 * 16 * 16, n, dtype=np.uint64)               # group index 2q + colour parity
    g[n // 2:] = rng.integers(0, 2**32, n - n // 2, dtype=np.uint64)   # and the full word range
    k0 = rng.integers(0, 2**32, n, dtype=np.uint64)
    k1 = rng.integers(0, 2**32, n, dtype=np.uint64)
    inp = "\n".join(f"{a} {b} {c} {d} {e}" for a, b, c, d, e in zip(s, c1, g, k0, k1)) + "\n"
    out = subprocess.run([driver], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    rows = np.array([[int(x) for x in line.split()] for line in out if line.strip()], dtype=np.uint64)
    assert rows.shape == (n, 12)
    assert np.array_equal(rows[:, 0:4], rows[:, 4:8]), "philox_sweep_pre + philox_group_prod differs from philox10"
    assert np.array_equal(rows[:, 0:4], rows[:, 8:12]), "philox_pre + philox_slot differs from philox10"
    for i in range(0, n, 8):                                           # the plain form against the oracle
        ref = oracle.philox4x32_10([s[i], c1[i], g[i], 0], [k0[i], k1[i]])
        assert [int(x) for x in ref] == [int(x) for x in rows[i, 0:4]], i
