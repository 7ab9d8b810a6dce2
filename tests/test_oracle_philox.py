"""Pins of the oracle's Philox4x32-10 generator (Salmon et al., SC'11)."""
import os

import numpy as np

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        w = [int(t, 16) for t in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_known_answer_vectors():
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, out in rows:
        assert oracle.philox(ctr, key) == out


def test_uniform_histogram():
    # 24-bit uniforms from consecutive counters are uniform on [0,1):
    # chi-square over 64 bins, 2^16 draws (4 per call).
    key = [12345, 678]
    u = []
    for i in range(1 << 14):
        u += [oracle.lib().orc_u01(v) for v in oracle.philox([i, 7, 3, 1], key)]
    u = np.array(u)
    assert u.min() >= 0 and u.max() < 1
    h, _ = np.histogram(u, bins=64, range=(0, 1))
    e = len(u) / 64
    chi2 = ((h - e) ** 2 / e).sum()
    assert chi2 < 120  # 63 dof: P(chi2 > 120) ~ 1e-5
