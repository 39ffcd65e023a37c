"""Moving lattice on the GPU against the oracle (positions, velocities,
spins, electron temperatures), energy conservation, observables, and the
full 40^3 bcc-Fe size."""
import numpy as np
import pytest

import oracle as O
import paper_2608_18541_b300 as P
from paper_2608_18541_b300 import workloads as W

pytestmark = pytest.mark.gpu

FS = 1e-15


def _case(n=6, T=300.0, alpha=0.1, ttm=True):
    s = W.bcc_fe(n, T=T, alpha=alpha)
    lat = W.morse_fe_lattice(T_init=300.0)
    t = W.ttm_z_exp((2, 2, 4), 1200.0, 40 * FS, 0.25, Lz=n * 2.8665) if ttm else None
    return s, t, lat


def _compare(g, o, tol_pos, tol_vel, tol_spin, L=6 * 2.8665):
    dx = g.get_positions() - o.positions()
    dx -= np.round(dx / L) * L          # both wrap into the box; compare modulo L
    assert np.abs(dx).max() <= tol_pos, np.abs(dx).max()
    v = o.velocities()
    assert np.abs(g.get_velocities() - v).max() <= tol_vel * np.abs(v).max()
    assert np.abs(g.get_spins() - o.spins()).max() <= tol_spin


@pytest.mark.parametrize("precision,tol", [(64, (1e-9, 1e-9, 1e-10)), (32, (2e-4, 2e-3, 2e-5))])
def test_moving_lattice_parity(precision, tol):
    s, t, lat = _case()
    g = P.System(s, t, precision=precision, lattice=lat)
    o = O.Oracle(s, t, lattice=lat)
    assert g.engine_now() == "general"
    for chunk in (1, 4, 10):
        g.step(chunk)
        o.lattice_step(chunk)
        _compare(g, o, *tol)
    Te, _, P0 = g.get_ttm(0, 16)
    assert abs(P0 - o.P0) <= 1e-9 * o.P0
    assert np.allclose(Te, o.ttm()[0], rtol=1e-9 if precision == 64 else 1e-5)
    g.sync()


def test_moving_lattice_energy_conservation_matches_oracle():
    s = W.bcc_fe(6, T=0.0, alpha=0.0, B=0.5)
    s["K"] = [0.0]
    s["sample_every"] = 10
    lat = W.morse_fe_lattice(T_init=300.0, gamma_p=0.0)
    g = P.System(s, None, precision=64, lattice=lat)
    o = O.Oracle(s, None, lattice=lat)
    g.step(100)
    o.lattice_step(100)
    gs, os_ = g.observables(0), o.samples()
    assert gs.shape == os_.shape == (10, P.NOBS)
    for k in (10, 12, 16, 17, 18):
        assert np.allclose(gs[:, k], os_[:, k], rtol=1e-8, atol=1e-12 * np.abs(os_[:, k]).max()), k
    etot = gs[:, 10] + gs[:, 11] + gs[:, 12] + gs[:, 17] + gs[:, 18]
    assert np.abs(etot - etot[0]).max() < 1e-3 * gs[:, 17].mean()


def test_full_size_moving_fe_40():
    s, t, lat = W.config_moving_fe(40)
    t = dict(t, source="power", P0=2e21)      # a given source power: no calibration run
    s["dt"] = 0.1 * FS
    g = P.System(s, t, precision=32, lattice=lat)
    assert g.n_total == 128000
    g.step(2)
    g.sync()
    o = O.Oracle(s, t, lattice=lat)
    o.lattice_step(2)
    dx = g.get_positions() - o.positions()
    L = 40 * 2.8665
    dx -= np.round(dx / L) * L
    assert np.abs(dx).max() < 2e-4
    assert np.abs(g.get_spins() - o.spins()).max() < 2e-5


def test_moving_lattice_checkpoint_resume_is_bitwise():
    s, t, lat = _case(n=6)
    a = P.System(s, t, precision=32, lattice=lat)
    a.step(3)
    blob = a.get_state()
    a.step(4)
    b = P.System(s, t, precision=32, lattice=lat)
    b.set_state(blob)
    b.step(4)
    assert np.array_equal(a.get_spins(), b.get_spins())
    assert np.array_equal(a.get_positions(), b.get_positions())
    assert np.array_equal(a.get_velocities(), b.get_velocities())
    assert np.array_equal(a.get_ttm(0, 16)[0], b.get_ttm(0, 16)[0])
