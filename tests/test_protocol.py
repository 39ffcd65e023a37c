"""Host-side switching statistics (paper Sec. II.G) and the step-profile
bath of the oracle (Sec. II.D)."""
import numpy as np
import pytest

import oracle as O
from paper_2608_18541_b300 import protocol as PR
from paper_2608_18541_b300 import workloads as W

FS = 1e-15


def test_wilson_interval_matches_the_paper_and_limits():
    # the paper quotes 20/20 switching with the Wilson 95 % CI [0.84, 1.00]
    lo, hi = PR.wilson_interval(20, 20)
    assert round(lo, 2) == 0.84 and hi == 1.0
    # symmetric under k -> n - k, and it contains the point estimate
    for k, n in [(3, 20), (10, 20), (17, 40)]:
        a, b = PR.wilson_interval(k, n)
        c, d = PR.wilson_interval(n - k, n)
        assert abs(a - (1 - d)) < 1e-12 and abs(b - (1 - c)) < 1e-12
        assert a < k / n < b
    # large n: the normal-approximation half width
    a, b = PR.wilson_interval(5000, 10000)
    assert abs((b - a) / 2 - 1.96 * 0.5 / 100) < 1e-4


def test_switching_criterion():
    t = np.arange(10) * 1.0
    rows = np.zeros((10, 20))
    rows[:, 0] = t
    rows[:, 6] = [-1, -0.5, 0.2, 0.4, -0.1, 0.3, 0.5, 0.6, 0.7, 0.8]
    assert PR.gd_switched(rows, t_cool_end=5.0)          # reversed from t = 5 on
    assert not PR.gd_switched(rows, t_cool_end=4.0)      # not yet at t = 4
    assert not PR.gd_switched(rows, t_cool_end=20.0)     # no rows after the stage


def test_oracle_step_profile_is_the_closed_form():
    sysd = W.gdfeco_fcc(2, sample_every=1)
    bath = {"cells": [1, 1, 1], "gamma_e": 225.0, "C_l": 3.1e6, "G": 0.0, "kappa_e": 0.0, "T0": 300.0,
            "source": "step_profile", "peak_Te": 1100.0, "fwhm": 3.0 * sysd["dt"], "t0": 4.0 * sysd["dt"],
            "spatial": "uniform"}
    o = O.Oracle(sysd, bath)
    assert o.ttm()[0][0] == 1100.0                       # t = 0 is in the first stage
    o.step(12)
    rows = o.samples()
    want = [1100.0 if (k + 1) < 4 else (550.0 if (k + 1) < 7 else 300.0) for k in range(12)]
    assert np.array_equal(rows[:, 15], want)
    assert np.array_equal(rows[:, 16], [300.0] * 12)


def test_fcc_gdfeco_model():
    o = O.Oracle(W.gdfeco_fcc(3))
    sp = o.species()
    assert o.n == 4 * 27 and sp.sum() == round(0.25 * o.n)
    assert o.ncolours == 4                                 # basis colouring
    # every atom has its 12 nearest neighbours at a / sqrt(2) and no others
    counts = [len(o.neighbours(i)[0]) for i in range(o.n)]
    assert set(counts) == {12}


def test_t90_of_a_closed_form_relaxation():
    from paper_2608_18541_b300 import threetemp as TT
    t = np.linspace(0.0, 10.0, 10001)
    T = 300.0 + 500.0 * (1.0 - np.exp(-t / 1.5))
    # exact: 1 - exp(-t/tau) = 0.9 * (1 - exp(-10/tau)) for the tail-mean final value
    Tf = T[-1000:].mean()
    frac = 0.9 * (Tf - 300.0) / 500.0
    want = -1.5 * np.log(1.0 - frac)
    assert abs(TT.t90(t, T) - want) < 2e-3
    assert abs(TT.t90(t, 1000.0 - (T - 300.0)) - want) < 2e-3      # a falling curve
