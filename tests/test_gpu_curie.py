"""Per-instance bath temperatures: a batched temperature scan of bcc Fe (the
<|m|>(T) curve of the Curie-temperature test, paper Sec. III) advances every
temperature in one system.  The FP64 state matches the oracle instance by
instance; the FP32 <|m|> falls with T and agrees with the FP64 oracle's."""
import numpy as np
import pytest

import oracle as O
import paper_2608_18541_b300 as P
from paper_2608_18541_b300 import workloads as W

pytestmark = pytest.mark.gpu

TEMPS = [100.0, 400.0, 700.0, 1000.0, 1300.0, 1600.0]


def _absm(s):
    return np.linalg.norm(s.mean(0))


def test_instance_bath_temperatures_match_oracle_exactly():
    sysd = W.curie_scan([150.0, 900.0], n=4, reps=1)
    g = P.System(sysd, precision=64, engine="general")
    g.step(25)
    for i in range(2):
        o = O.Oracle(sysd, instance=i, index=i)
        o.step(25)
        assert np.abs(g.get_spins(i) - o.spins()).max() <= 1e-10
        assert np.isclose(g.observe_now(i)[15], [150.0, 900.0][i])


def test_magnetisation_falls_with_temperature_and_matches_oracle():
    reps = 2
    sysd = W.curie_scan(TEMPS, n=6, reps=reps)
    g = P.System(sysd, precision=32, engine="general")
    g.step(300)
    acc = np.zeros(len(TEMPS) * reps)
    nsamp = 10
    for _ in range(nsamp):
        g.step(30)
        acc += [_absm(g.get_spins(i)) for i in range(len(acc))]
    m = (acc / nsamp).reshape(len(TEMPS), reps).mean(1)
    assert m[0] > 0.85, m
    assert all(m[k + 1] < m[k] + 0.02 for k in range(len(m) - 1)), m
    assert m[-1] < m[0] - 0.3, m
    # FP64 oracle, same realisations, at one temperature mid-curve
    k = 2
    om = 0.0
    for r in range(reps):
        i = k * reps + r
        o = O.Oracle(sysd, instance=i, index=i)
        o.step(300)
        for _ in range(nsamp):
            o.step(30)
            om += _absm(o.spins())
    om /= reps * nsamp
    assert abs(om - m[k]) < 0.03, (om, m[k])
