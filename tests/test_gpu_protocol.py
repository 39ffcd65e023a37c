"""The paper's GdFeCo protocol on the GPU: fcc lattice, Bethe-Slater exchange
re-derived for fcc, the three-stage step profile of T_e (Sec. II.D) with a
per-instance peak and cooling stage, against the oracle state by state; and
the switching statistics of a small campaign (Sec. II.G)."""
import numpy as np
import pytest

import oracle as O
import paper_2608_18541_b300 as P
from paper_2608_18541_b300 import protocol as PR
from paper_2608_18541_b300 import workloads as W

pytestmark = pytest.mark.gpu
FS = 1e-15
TOL = {64: 1e-10, 32: 2e-5}


@pytest.mark.parametrize("precision,sweep", [(64, "symmetric"), (32, "symmetric"), (64, "merged")])
def test_step_profile_fcc_gdfeco_matches_oracle(precision, sweep):
    dt = 0.2 * FS
    sysd, bath, _ = W.switching_campaign([900.0, 1800.0], [1, 3], reps=1, n=3, t_peak=10 * dt, t_cool=8 * dt,
                                         t_tail=20 * dt, sample_every=7)
    sysd = dict(sysd, sweep=sweep)
    g = P.System(sysd, bath, precision=precision, engine="general")
    assert g.info().max_colours == 4
    calls = (9, 31, 40)           # the merged sweep closes at the end of every call: same calls on both sides
    for n in calls:
        g.step(n)
    for i in range(4):
        o = O.Oracle(sysd, bath, instance=i, index=i)
        for n in calls:
            o.step(n)
        assert np.abs(g.get_spins(i) - o.spins()).max() <= TOL[precision], i
        gs, osm = g.observables(i), o.samples()
        assert np.array_equal(gs[:, 15], osm[:, 15])        # the prescribed T_e, step by step
        assert np.allclose(gs[:, 1:7], osm[:, 1:7], atol=10 * TOL[precision])


def test_small_switching_campaign_runs_and_reports():
    # fcc 6^3 (864 atoms) x 2 peaks x 2 cooling multipliers x 4 realisations:
    # the statistics machinery end to end (not the paper's numbers)
    sysd, bath, steps = W.switching_campaign([1100.0, 2600.0], [2, 6], reps=4, n=6, t_peak=300 * FS,
                                             t_cool=300 * FS, t_tail=500 * FS, dt=1.0 * FS, sample_every=20)
    g = P.System(sysd, bath, precision=32)
    g.step(steps)
    res = {}
    for k, inst in enumerate(sysd["instances"]):
        rows = g.observables(k)
        t_end = bath["t0"] + inst["fwhm"]
        res.setdefault((inst["peak_Te"], inst["fwhm"]), []).append(PR.gd_switched(rows, t_end))
        # demagnetised during the peak stage, sign of Fe m_z recorded every 20 steps
        assert rows[:, 3].min() < 0.8
    for key, v in res.items():
        lo, hi = PR.wilson_interval(sum(v), len(v))
        assert 0.0 <= lo <= sum(v) / len(v) <= hi <= 1.0
