"""GPU path against the oracle, element by element, through the C ABI.

Tolerances (spec bar): FP64 spins within 1e-10 per component and FP32
spins within 2e-5 per component of the FP64 oracle over the first 200 steps;
integer set-up (species placement, colour classes) bit-exact; TTM grids and
observables in FP64 within 1e-10 relative.
"""
import numpy as np
import pytest

import oracle as O
import paper_2608_18541_b300 as P
from paper_2608_18541_b300 import workloads as W

pytestmark = pytest.mark.gpu

FS = 1e-15
TOL = {64: 1e-10, 32: 2e-5}


def _pair(sysd, ttm=None, precision=64, engine="general", inst=0, gpu=None):
    g = gpu or P.System(sysd, ttm, precision=precision, engine=engine)
    o = O.Oracle(sysd, ttm, instance=inst)
    assert np.array_equal(g.get_species(inst), o.species())
    assert np.array_equal(g.get_colours(inst), o.colours())
    return g, o


def _compare_spins(g, o, precision, inst=0):
    d = np.abs(g.get_spins(inst) - o.spins()).max()
    assert d <= TOL[precision], d
    return d


CASES = {
    "bcc_fe_10": lambda: (W.config_bcc_fe_2000(), None),
    "gdfeco_32_ttm": lambda: W.config_gdfeco_32(),
    "gdfeco_11_odd": lambda: (W.gdfeco_sc(11, T=500.0, B=0.5), None),
    "bcc_fe_5_greedy": lambda: (W.bcc_fe(5, T=600.0), None),
    "gdfeco_12_spot": lambda: (W.gdfeco_sc(12), W.ttm_xy_spot(4, 1800.0, 20 * FS, sigma_xy=10.0)),
}


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("case", sorted(CASES))
def test_exact_state_200_steps(case, precision):
    sysd, ttm = CASES[case]()
    g, o = _pair(sysd, ttm, precision)
    for chunk in (1, 49, 150):
        g.step(chunk)
        o.step(chunk)
        _compare_spins(g, o, precision)
    g.sync()
    assert g.get_step() == 200
    if ttm is not None:
        nc = int(np.prod(ttm["cells"]))
        Te, Tl, P0 = g.get_ttm(0, nc)
        oTe, oTl = o.ttm()
        assert abs(P0 - o.P0) <= 1e-9 * o.P0
        assert np.allclose(Te, oTe, rtol=1e-10, atol=0)
        assert np.allclose(Tl, oTl, rtol=1e-10, atol=0)


@pytest.mark.parametrize("precision", [64, 32])
def test_batched_instances_of_uneven_size(precision):
    sysd, ttm = W.config_ensemble(n_peak=2, n_dur=2, n_real=2, lmin=6, lmax=9)
    g = P.System(sysd, ttm, precision=precision, engine="general")
    assert g.n_instances == 8
    g.step(60)
    for inst in range(g.n_instances):
        o = O.Oracle(sysd, ttm, instance=inst)
        assert np.array_equal(g.get_species(inst), o.species())
        o.step(60)
        _compare_spins(g, o, precision, inst)
        Te, Tl, P0 = g.get_ttm(inst, 1)
        assert abs(P0 - o.P0) <= 1e-9 * o.P0
        assert np.allclose(Te, o.ttm()[0], rtol=1e-10)


def test_explicit_cluster():
    rng = np.random.default_rng(3)
    pos = rng.uniform(0, 12, size=(40, 3))
    sysd = W.cluster(pos, J=2e-21, rc=3.2, mu=2.0, B=(0.1, 0.0, 1.0), T=50.0, alpha=0.2, dt=0.2 * FS, K=1e-23)
    g, o = _pair(sysd, None, 64)
    g.step(200)
    o.step(200)
    _compare_spins(g, o, 64)


def test_observable_samples_match():
    sysd = W.gdfeco_sc(10, sample_every=10)
    ttm = W.ttm_single_cell(1200.0, 20 * FS)
    g, o = _pair(sysd, ttm, 64)
    g.step(100)
    o.step(100)
    gs, os_ = g.observables(0), o.samples()
    assert gs.shape == os_.shape == (10, P.NOBS)
    assert np.array_equal(gs[:, 19], os_[:, 19])
    scale = np.maximum(np.abs(os_), 1e-30)
    fields = [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16]
    err = np.abs(gs[:, fields] - os_[:, fields]) / np.maximum(scale[:, fields], 1e-12 * np.abs(os_[:, fields]).max(0))
    assert err.max() < 1e-9, err.max(0)
    now = g.observe_now(0)
    ref = o.observe()
    assert np.allclose(now[:17], ref[:17], rtol=1e-9, atol=1e-12 * np.abs(ref[:17]).max())


def test_checkpoint_resume_is_bitwise():
    sysd, ttm = W.config_gdfeco_32()
    sysd = dict(sysd, sample_every=25)
    a = P.System(sysd, ttm, precision=32)
    a.step(50)
    blob = a.get_state()
    a.step(50)
    end_a = a.get_spins()
    b = P.System(sysd, ttm, precision=32)
    b.set_state(blob)
    b.step(50)
    assert np.array_equal(b.get_spins(), end_a)
    assert np.array_equal(b.observables(0), a.observables(0))


def test_run_to_run_bitwise():
    sysd, ttm = W.config_gdfeco_32()
    out = []
    for _ in range(2):
        g = P.System(sysd, ttm, precision=32)
        g.step(30)
        out.append(g.get_spins())
    assert np.array_equal(out[0], out[1])


def test_non_finite_state_sets_the_health_flag():
    # a NaN written into the state on the host (not through set_spins, which
    # rejects it) is caught by the device health word after the next step
    sysd = W.gdfeco_sc(6)
    g = P.System(sysd, precision=64, engine="general")
    blob = bytearray(g.get_state())
    hdr = 8 * 8
    blob[hdr:hdr + 8] = np.array([np.nan]).tobytes()
    g.set_state(bytes(blob))
    g.step(1)
    with pytest.raises(P.TTSError) as ei:
        g.sync()
    assert ei.value.code == -5


def test_set_get_spins_roundtrip_normalises():
    sysd = W.bcc_fe(4)
    g = P.System(sysd, precision=64)
    rng = np.random.default_rng(1)
    s = rng.normal(size=(g.n_total, 3)) * 3.0
    g.set_spins(s)
    back = g.get_spins()
    assert np.allclose(back, s / np.linalg.norm(s, axis=1, keepdims=True), atol=1e-15)
    with pytest.raises(P.TTSError):
        g.set_spins(np.zeros((g.n_total, 3)))
