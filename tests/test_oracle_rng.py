"""Oracle pins: counter-based noise (Philox4x32-10, uniforms, Box-Muller)."""
import os

import numpy as np
import pytest
from scipy import stats

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(x, 16) for x in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat_rows())
def test_philox_known_answers(ctr, key, out):
    assert O.philox(ctr, key) == out


def test_uniform_endpoints_and_exactness():
    # ((x >> 9) + 0.5) * 2^-23: strictly inside (0, 1), symmetric, and exactly
    # representable in float32 (so both precisions see the same value)
    assert O.uniform(0) == 2.0 ** -24
    assert O.uniform(0xffffffff) == 1.0 - 2.0 ** -24
    assert O.uniform(0x000001ff) == O.uniform(0)
    assert O.uniform(0x00000200) == 3 * 2.0 ** -24
    for x in (0, 1 << 9, 12345678, 0xdeadbeef, 0xfffffe00, 0xffffffff):
        u = O.uniform(x)
        assert float(np.float32(u)) == u
        assert 0.0 < u < 1.0


def _draws(n):
    key = (42, 0)
    g = np.empty((n, 3))
    for i in range(n):
        w = O.philox((i, 7, 3, 1), key)
        g[i] = O.gauss3(w)
    return g


def test_box_muller_normal_moments_and_independence():
    g = _draws(60000)
    flat = g.reshape(-1)
    n = flat.size
    assert abs(flat.mean()) < 5 * np.sqrt(1.0 / n)
    assert abs(flat.var() - 1.0) < 5 * np.sqrt(2.0 / n)
    assert abs(stats.kurtosis(flat, fisher=False) - 3.0) < 5 * np.sqrt(24.0 / n)
    assert abs(stats.skew(flat)) < 5 * np.sqrt(6.0 / n)
    # each of the three components is standard normal on its own
    for k in range(3):
        assert stats.kstest(g[:, k], "norm").pvalue > 1e-4
    # components uncorrelated (g1, g2 share a radius but are independent)
    c = np.corrcoef(g.T)
    m = g.shape[0]
    for a in range(3):
        for b in range(a + 1, 3):
            assert abs(c[a, b]) < 5 / np.sqrt(m)
    # g1^2 + g2^2 is chi-square with 2 degrees of freedom (pins the shared radius)
    assert stats.kstest(g[:, 0] ** 2 + g[:, 1] ** 2, "chi2", args=(2,)).pvalue > 1e-4


def test_box_muller_values_from_uniforms():
    # g1 = sqrt(-2 ln u0) cos(2 pi u1) for chosen words: with u1 = 1/4 + 2^-24
    # the cosine is ~0 and the sine ~1, with u1 = 1/2 + 2^-24 the cosine is ~-1
    x_quarter = (1 << 30)           # ((2^21)+0.5) 2^-23 = 1/4 + 2^-24
    x_half = (1 << 31)
    x_e = int((np.exp(-0.5) * 2 ** 23 - 0.5)) << 9   # u0 ~ e^-1/2 -> radius ~ 1
    u0 = O.uniform(x_e)
    r = np.sqrt(-2 * np.log(u0))
    g = O.gauss3([x_e, x_quarter, x_e, x_half])
    assert abs(g[0] - r * np.cos(2 * np.pi * (0.25 + 2 ** -24))) < 1e-15
    assert abs(g[1] - r) < 1e-12
    assert abs(g[2] + r) < 1e-12
