"""Three-temperature relaxation of moving-lattice bcc Fe on the GPU (the
paper's Sec. III benchmark): hot electrons on one uniform cell cool into the
lattice through the electron-ion friction while the spins heat up; the
lattice equilibration time falls as the friction grows.  The same path is
parity-tested against the oracle in test_gpu_lattice.py."""
import numpy as np
import pytest

import paper_2608_18541_b300 as P
from paper_2608_18541_b300 import threetemp as TT
from paper_2608_18541_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _run(gamma_scale, steps=1200):
    s, bath, lat = W.three_temperature(10, gamma_scale)
    g = P.System(s, bath, precision=32, lattice=lat, obs_capacity=steps // 25 + 2)
    g.set_ttm_state([900.0], [300.0])
    g.step(steps)
    return TT.temperatures(g.observables(0))


def test_three_temperatures_converge_and_t90_falls_with_friction():
    res = {gs: _run(gs) for gs in (4.0, 8.0, 16.0)}
    t90 = {}
    for gs, (t, Te, Tl, Ts) in res.items():
        assert Te[0] > 600.0 and Te[-1] < Te[0]             # electrons cool
        assert Tl[-1] > Tl[0] + 20.0                        # the lattice heats
        assert Ts[-1] > 100.0                               # the spins heat (from 0 K)
        t90[gs] = TT.t90(t, Tl)
    assert t90[4.0] > t90[8.0] > t90[16.0], t90
    t, Te, Tl, Ts = res[16.0]
    k = len(t) // 10
    assert abs(Te[-k:].mean() - Tl[-k:].mean()) < 0.1 * Te[-k:].mean()   # electrons and lattice meet


def test_colour_margin_matches_oracle_and_keeps_parity():
    """colour_rc: no two atoms within 4.9 A share a colour (greedy, the bcc
    rule no longer qualifies); the colours are bit-identical to the oracle's
    and a moving-lattice run matches it."""
    import oracle as O
    s, bath, lat = W.three_temperature(6, 4.0, sample_every=5)
    g = P.System(s, bath, precision=64, lattice=lat)
    o = O.Oracle(s, bath, lattice=lat)
    assert np.array_equal(g.get_colours(), o.colours())
    assert g.info().max_colours == o.ncolours > 4
    for sys_ in (g, o):
        sys_.set_ttm_state(np.array([1200.0]), np.array([300.0]))
    g.step(40)
    o.lattice_step(40)
    assert np.abs(g.get_spins() - o.spins()).max() <= 1e-9
    assert np.allclose(g.get_ttm()[0], o.ttm()[0], rtol=1e-9)
