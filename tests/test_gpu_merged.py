"""Merged (leapfrog) sweep on the GPU against the oracle's merged mode:
every engine, both precisions, with sampling and several calls (the sweep
closes at sampling steps and at the end of every call on both sides).  Same
bar as the symmetric sweep: FP64 within 1e-10, FP32 within 2e-5 per spin
component."""
import numpy as np
import pytest

import oracle as O
import paper_2608_18541_b300 as P
from paper_2608_18541_b300 import workloads as W

pytestmark = pytest.mark.gpu

FS = 1e-15
TOL = {64: 1e-10, 32: 2e-5}
CALLS = (1, 37, 50, 112)


def _merged(sysd):
    return dict(sysd, sweep="merged")


def _compare(g, sysd, ttm, precision, ninst=1, base=0):
    os_ = [O.Oracle(sysd, ttm, instance=base + i, index=i) for i in range(ninst)]
    for n in CALLS:
        g.step(n)
        for o in os_:
            o.step(n)
        for i, o in enumerate(os_):
            d = np.abs(g.get_spins(i) - o.spins()).max()
            assert d <= TOL[precision], (n, i, d)
    return os_


@pytest.mark.parametrize("precision", [64, 32])
def test_checker_merged_matches_oracle(precision):
    sysd = _merged(W.gdfeco_sc(16, sample_every=25))
    ttm = W.ttm_single_cell(1500.0, 20 * FS)
    g = P.System(sysd, ttm, precision=precision, engine="checker")
    assert g.engine == "checker"
    os_ = _compare(g, sysd, ttm, precision)
    gs, osm = g.observables(0), os_[0].samples()
    assert gs.shape == osm.shape
    assert np.array_equal(gs[:, 19], osm[:, 19])
    assert np.allclose(gs[:, 1:7], osm[:, 1:7], atol=TOL[precision] * 10)


def test_checker_merged_grid_instances_and_every_config():
    sysd = _merged(W.gdfeco_sc(16))
    sysd["instances"] = [{"nx": 16, "ny": 16, "nz": 16, "frac1": f} for f in (0.2, 0.3)]
    ttm = W.ttm_xy_spot(4, 1800.0, 20 * FS, sigma_xy=12.0)
    g = P.System(sysd, ttm, precision=32, engine="checker")
    _, n = g.set_config(-1)
    state = g.get_state()
    ref = None
    for c in range(n):
        g.set_state(state)
        g.set_config(c)
        g.step(30)
        spins = [g.get_spins(i) for i in range(2)]
        if ref is None:
            ref = spins
            for i in range(2):
                o = O.Oracle(sysd, ttm, instance=i, index=i)
                o.step(30)
                assert np.abs(spins[i] - o.spins()).max() <= TOL[32]
        else:
            for a, b in zip(ref, spins):
                assert np.array_equal(a, b), c


@pytest.mark.parametrize("precision", [64, 32])
def test_general_merged_matches_oracle(precision):
    sysd = _merged(W.bcc_fe(4))
    g = P.System(sysd, precision=precision, engine="general")
    assert g.info().max_colours == 4
    _compare(g, sysd, None, precision)


@pytest.mark.parametrize("precision", [64, 32])
def test_resident_merged_matches_oracle_mixed_colour_counts(precision):
    sysd, ttm = W.config_ensemble(n_peak=1, n_dur=2, n_real=2, lmin=7, lmax=10)
    sysd = _merged(sysd)
    g = P.System(sysd, ttm, precision=precision, engine="resident")
    assert g.engine == "resident"
    _compare(g, sysd, ttm, precision, ninst=len(sysd["instances"]))


def test_merged_general_needs_one_colour_count():
    sysd = _merged(W.gdfeco_sc(6))
    sysd["instances"] = [{"nx": 6, "ny": 6, "nz": 6, "frac1": 0.25}, {"nx": 7, "ny": 7, "nz": 7, "frac1": 0.25}]
    g = P.System(sysd, precision=64, engine="general")
    with pytest.raises(P.TTSError):
        g.step(3)


@pytest.mark.parametrize("sweep", ["symmetric", "merged"])
def test_resident_call_longer_than_a_bath_chunk(sweep):
    """The resident engine advances a call in chunks of at most 256 steps (the
    bath trajectory of every instance first, then the spins): a 300-step call
    with sampling matches the oracle, the merged sweep staying open across
    the chunk boundary."""
    sysd, ttm = W.config_ensemble(n_peak=1, n_dur=1, n_real=3, lmin=5, lmax=8)
    sysd = dict(sysd, sweep=sweep, sample_every=40)
    g = P.System(sysd, ttm, precision=64, engine="resident")
    assert g.engine == "resident"
    g.step(300)
    for i in range(3):
        o = O.Oracle(sysd, ttm, instance=i, index=i)
        o.step(300)
        assert np.abs(g.get_spins(i) - o.spins()).max() <= TOL[64]
        gs, osm = g.observables(i), o.samples()
        assert np.array_equal(gs[:, 19], osm[:, 19])
        assert np.allclose(gs[:, 15], osm[:, 15], rtol=1e-10)
        assert np.allclose(gs[:, 1:7], osm[:, 1:7], atol=1e-9)
