"""Fast engines (checkerboard, resident) against the oracle, and at the full
sizes of the benchmark's launch configurations.

Same bar as the general engine: FP64 within 1e-10, FP32 within 2e-5 per spin
component over 200 steps; bit-exact integer set-up.
"""
import numpy as np
import pytest

import oracle as O
import paper_2608_18541_b300 as P
from paper_2608_18541_b300 import workloads as W

pytestmark = pytest.mark.gpu

FS = 1e-15
TOL = {64: 1e-10, 32: 2e-5}


def _check_instance(g, sysd, ttm, inst, steps_done, precision, ncells=1):
    o = O.Oracle(sysd, ttm, instance=inst)
    assert np.array_equal(g.get_species(inst), o.species())
    assert np.array_equal(g.get_colours(inst), o.colours())
    o.step(steps_done)
    d = np.abs(g.get_spins(inst) - o.spins()).max()
    assert d <= TOL[precision], (inst, d)
    if ttm is not None:
        Te, Tl, P0 = g.get_ttm(inst, ncells)
        oTe, oTl = o.ttm()
        assert abs(P0 - o.P0) <= 1e-9 * o.P0
        assert np.allclose(Te, oTe, rtol=1e-10)
        assert np.allclose(Tl, oTl, rtol=1e-10)
    return o


@pytest.mark.parametrize("precision", [64, 32])
def test_checker_exact_state_gdfeco_32_ttm(precision):
    sysd, ttm = W.config_gdfeco_32()
    g = P.System(sysd, ttm, precision=precision, engine="checker")
    assert g.engine == "checker"
    o = O.Oracle(sysd, ttm)
    for chunk in (1, 99, 100):
        g.step(chunk)
        o.step(chunk)
        d = np.abs(g.get_spins() - o.spins()).max()
        assert d <= TOL[precision], d


@pytest.mark.parametrize("precision", [64, 32])
def test_checker_spatial_grid_and_instances(precision):
    sysd = W.gdfeco_sc(12)
    sysd["instances"] = [{"nx": 12, "ny": 12, "nz": 12, "frac1": f} for f in (0.2, 0.25, 0.3)]
    ttm = W.ttm_xy_spot(4, 1800.0, 20 * FS, sigma_xy=10.0)
    g = P.System(sysd, ttm, precision=precision, engine="checker", instance_base=5)
    g.step(200)
    for inst in range(3):
        o = O.Oracle(sysd, ttm, instance=5 + inst, index=inst)
        o.step(200)
        assert np.array_equal(g.get_species(inst), o.species())
        assert np.abs(g.get_spins(inst) - o.spins()).max() <= TOL[precision]
        Te, Tl, _ = g.get_ttm(inst, 64)
        assert np.allclose(Te, o.ttm()[0], rtol=1e-10)


@pytest.mark.parametrize("precision", [64, 32])
def test_resident_exact_state_odd_uniform_bath(precision):
    sysd = W.gdfeco_sc(11, T=500.0, B=0.5)
    g = P.System(sysd, precision=precision, engine="resident")
    assert g.engine == "resident"
    g.step(1)
    g.step(99)
    g.step(100)
    _check_instance(g, sysd, None, 0, 200, precision)


@pytest.mark.parametrize("precision", [64, 32])
def test_resident_batched_ensemble_with_pulses(precision):
    sysd, ttm = W.config_ensemble(n_peak=2, n_dur=2, n_real=3, lmin=6, lmax=13)
    g = P.System(sysd, ttm, precision=precision, engine="resident")
    assert g.engine == "resident" and g.n_instances == 12
    g.step(120)
    g.step(80)
    for inst in range(g.n_instances):
        _check_instance(g, sysd, ttm, inst, 200, precision)


@pytest.mark.parametrize("engine", ["checker", "resident"])
def test_engine_observables_match_oracle(engine):
    sysd = W.gdfeco_sc(10, sample_every=10)
    ttm = W.ttm_single_cell(1200.0, 20 * FS)
    g = P.System(sysd, ttm, precision=64, engine=engine)
    assert g.engine == engine
    o = O.Oracle(sysd, ttm)
    g.step(100)
    o.step(100)
    gs, os_ = g.observables(0), o.samples()
    assert gs.shape == os_.shape == (10, P.NOBS)
    assert np.array_equal(gs[:, 19], os_[:, 19])
    for k in range(17):
        scale = max(np.abs(os_[:, k]).max(), 1e-300)
        assert np.abs(gs[:, k] - os_[:, k]).max() <= 1e-9 * scale, k


@pytest.mark.parametrize("engine", ["checker", "resident"])
def test_engine_checkpoint_resume_is_bitwise(engine):
    sysd, ttm = W.config_gdfeco_32()
    if engine == "resident":
        sysd = W.gdfeco_sc(12)
    sysd = dict(sysd, sample_every=25)
    a = P.System(sysd, ttm, precision=32, engine=engine)
    a.step(50)
    blob = a.get_state()
    a.step(50)
    end_a = a.get_spins()
    b = P.System(sysd, ttm, precision=32, engine=engine)
    b.set_state(blob)
    b.step(50)
    assert np.array_equal(b.get_spins(), end_a)
    assert np.array_equal(b.observables(0), a.observables(0))


def test_auto_engine_choice():
    assert P.System(W.bcc_fe(4), precision=32).engine == "general"
    s, t = W.config_ensemble(n_peak=1, n_dur=1, n_real=8, lmin=6, lmax=9)
    assert P.System(s, t, precision=32).engine == "resident"
    s, t = W.config_gdfeco_32()
    assert P.System(s, t, precision=32).engine == "checker"
    s = W.gdfeco_sc(11)
    assert P.System(s, precision=32).engine == "resident"
    # a multi-cell grid on a resident system hands over to the next valid engine
    g = P.System(s, precision=32)
    g.step(5)
    g.set_ttm_grid(W.ttm_xy_spot(4, 1500.0, 20 * FS, sigma_xy=10.0))
    assert g.engine_now() == "general"
    g.step(5)
    o = O.Oracle(s)
    o.step(5)
    o2 = O.Oracle(s, W.ttm_xy_spot(4, 1500.0, 20 * FS, sigma_xy=10.0))
    o2.set_spins(o.spins())
    o2.stepcount = 5
    o2.step(5)
    assert np.abs(g.get_spins() - o2.spins()).max() <= TOL[32]


def test_set_spins_reaches_the_engine():
    for engine in ("checker", "resident"):
        g = P.System(W.gdfeco_sc(8, T=0.0), precision=64, engine=engine)
        rng = np.random.default_rng(2)
        s = rng.normal(size=(g.n_total, 3))
        s /= np.linalg.norm(s, axis=1, keepdims=True)
        g.set_spins(s)
        g.step(3)
        o = O.Oracle(W.gdfeco_sc(8, T=0.0))
        o.set_spins(s)
        o.step(3)
        assert np.abs(g.get_spins() - o.spins()).max() < 1e-12


# ---------------------------------------------------------------------------
# full sizes, in the launch configurations the benchmark times
# ---------------------------------------------------------------------------
def test_full_size_gdfeco_128x4_checker_fp32():
    sysd, ttm = W.config_gdfeco_large(128, 4)
    g = P.System(sysd, ttm, precision=32, engine="auto")
    assert g.engine == "checker" and g.n_total == 4 * 128 ** 3
    g.step(3)
    # instance 0 calibrates the source in the oracle; instance 3 reuses that
    # oracle P0 (the calibration depends on the grid only, not on the alloy)
    o0 = _check_instance(g, sysd, ttm, 0, 3, 32, ncells=16 ** 3)
    ttm3 = dict(ttm, source="power", P0=o0.P0)
    o3 = O.Oracle(sysd, ttm3, instance=3)
    assert np.array_equal(g.get_species(3), o3.species())
    o3.step(3)
    assert np.abs(g.get_spins(3) - o3.spins()).max() <= TOL[32]
    s = g.get_all_spins()
    assert np.abs(np.linalg.norm(s, axis=1) - 1).max() < 1e-6


def test_full_size_ensemble_1024_resident_fp32():
    sysd, ttm = W.config_ensemble()
    g = P.System(sysd, ttm, precision=32, engine="auto")
    assert g.engine == "resident" and g.n_instances == 1024
    g.step(20)
    sizes = [n for n, _ in g.sizes]
    picks = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), 17, 511, 1023})
    for inst in picks:
        _check_instance(g, sysd, ttm, inst, 20, 32)


@pytest.mark.parametrize("engine,sysf", [
    ("checker", lambda: (W.gdfeco_sc(16), W.ttm_single_cell(1500.0, 20 * FS))),
    ("resident", lambda: W.config_ensemble(n_peak=1, n_dur=2, n_real=4, lmin=6, lmax=11)),
    ("general", lambda: (W.bcc_fe(6), None)),
])
def test_autotune_keeps_results_bitwise(engine, sysf):
    sysd, ttm = sysf()
    a = P.System(sysd, ttm, precision=32, engine=engine)
    a.step(30)
    b = P.System(sysd, ttm, precision=32, engine=engine)
    chosen, n = b.autotune(probe_steps=5)
    assert n >= 2 and 0 <= chosen < n
    assert b.get_step() == 0                 # the probes left no trace
    b.step(30)
    for i in range(a.n_instances):
        assert np.array_equal(a.get_spins(i), b.get_spins(i))


def _many_small_with_grid():
    """32 GdFeCo realisations of 16^3 with a 4^3 TTM grid each: more (column,
    z-plane) work units than the staged pass keeps CTAs, so a CTA marches over
    several planes and across column boundaries."""
    sysd = W.gdfeco_sc(16)
    sysd["instances"] = [{"nx": 16, "ny": 16, "nz": 16, "frac1": 0.25} for _ in range(32)]
    return sysd, W.ttm_xy_spot(4, 1500.0, sigma_xy=20.0)


@pytest.mark.parametrize("sysf", [
    lambda: (W.gdfeco_sc(16), W.ttm_single_cell(1500.0, 20 * FS)),
    _many_small_with_grid,
    lambda: (dict(W.gdfeco_sc(10), nx=16, ny=10, nz=12), W.ttm_single_cell(1200.0, 20 * FS)),
])
def test_every_checker_config_gives_the_same_spins(sysf):
    """The staged (shared-memory) pass and every block shape of the direct
    pass compute each site with the same arithmetic: bitwise equal spins."""
    sysd, ttm = sysf()
    g = P.System(sysd, ttm, precision=32, engine="checker")
    cur, n = g.set_config(-1)
    assert n >= 2 and cur == 0
    state = g.get_state()
    ref = None
    for c in range(n):
        g.set_state(state)
        assert g.set_config(c)[0] == c
        g.step(12)
        spins = [g.get_spins(i) for i in range(g.n_instances)]
        if ref is None:
            ref = spins
        else:
            for a, b in zip(ref, spins):
                assert np.array_equal(a, b), c
