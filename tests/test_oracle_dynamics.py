"""Oracle pins: the spin advance against closed forms of Eq. 1, an independent
ODE integration of Eq. 1, and exact conservation laws of the splitting."""
import numpy as np
import pytest
from scipy.integrate import solve_ivp

import oracle as O
from paper_2608_18541_b300 import workloads as W

GAMMA = 1.76085963023e11
MUB = 9.2740100783e-24
FS = 1e-15


def _tilted(theta_deg, phi_deg=0.0):
    t, p = np.radians(theta_deg), np.radians(phi_deg)
    return [np.sin(t) * np.cos(p), np.sin(t) * np.sin(p), np.cos(t)]


# ---------------------------------------------------------------------------
# single spin, exact
# ---------------------------------------------------------------------------
def test_larmor_precession_is_exact():
    B = 2.5
    sysd = W.single_spins(1, B=(0, 0, B), T=0.0, alpha=0.0, dt=1.0 * FS, init=_tilted(30))
    o = O.Oracle(sysd)
    assert o.ncolours == 1
    phis = []
    nstep = 400
    for _ in range(nstep):
        o.step(1)
        s = o.spins()[0]
        phis.append(np.arctan2(s[1], s[0]))
        assert abs(s[2] - np.cos(np.radians(30))) < 1e-14
    phi = np.unwrap(np.array(phis))
    t = np.arange(1, nstep + 1) * FS
    # counter-clockwise about +B at gamma B (Eq. 1 with alpha = 0)
    assert np.allclose(phi, GAMMA * B * t, rtol=1e-12, atol=0)


def test_damping_envelope_is_exact():
    B, alpha = 5.0, 0.1
    th0 = np.radians(70)
    sysd = W.single_spins(1, B=(0, 0, B), T=0.0, alpha=alpha, dt=2.0 * FS, init=_tilted(70))
    o = O.Oracle(sysd)
    for n in range(1, 301):
        o.step(1)
        t = n * 2.0 * FS
        exact = np.tanh(alpha * GAMMA * B * t / (1 + alpha ** 2) + np.arctanh(np.cos(th0)))
        assert abs(o.spins()[0][2] - exact) < 1e-13
    # azimuth advances at gamma B / (1 + alpha^2)
    s = o.spins()[0]
    phi = np.arctan2(s[1], s[0])
    want = (GAMMA * B / (1 + alpha ** 2) * 300 * 2.0 * FS) % (2 * np.pi)
    assert abs((phi - want + np.pi) % (2 * np.pi) - np.pi) < 1e-10


def test_anisotropy_kittel_frequency_is_exact():
    # K only, alpha = 0: field 2 K cos(theta) / mu along z, precession at
    # omega = gamma 2 K cos(theta) / mu (the paper's omega = (2K/hbar) cos theta
    # single-spin benchmark of Sec. III.A, in SI form)
    K = 5.0384e-5 * 1.602176634e-19
    mu = 2.2
    th = 20.0
    sysd = W.single_spins(1, mu=mu, B=(0, 0, 0), T=0.0, alpha=0.0, dt=0.5 * FS, K=K, init=_tilted(th))
    o = O.Oracle(sysd)
    phis = []
    for _ in range(500):
        o.step(1)
        s = o.spins()[0]
        phis.append(np.arctan2(s[1], s[0]))
    omega = GAMMA * 2 * K * np.cos(np.radians(th)) / (mu * MUB)
    phi = np.unwrap(phis)
    t = np.arange(1, 501) * 0.5 * FS
    assert np.allclose(phi, omega * t, rtol=1e-12, atol=1e-15)


def test_flow_map_properties():
    rng = np.random.default_rng(0)
    for _ in range(200):
        s = rng.normal(size=3)
        s /= np.linalg.norm(s)
        B = rng.normal(size=3) * 100
        s1 = O.flow(s, B, 0.0, 1e-15)
        assert abs(np.linalg.norm(s1) - 1) < 1e-15
        bh = B / np.linalg.norm(B)
        assert abs(s1 @ bh - s @ bh) < 1e-14           # alpha = 0 keeps the cone
        s2 = O.flow(s, B, 0.5, 1e-15)
        assert s2 @ bh >= s @ bh - 1e-15              # damping pulls toward +B
    # along the field nothing moves, antiparallel is a (unstable) fixed point too
    assert np.array_equal(O.flow([0, 0, 1.0], [0, 0, 3.0], 0.3, 1e-14), [0, 0, 1.0])
    assert np.array_equal(O.flow([0, 0, -1.0], [0, 0, 3.0], 0.3, 1e-14), [0, 0, -1.0])


# ---------------------------------------------------------------------------
# clusters: independent ODE integration of Eq. 1, second order of the sweep
# ---------------------------------------------------------------------------
def _llg_rhs_factory(pos, J, rc, mu, K, axis, B, alpha):
    n = len(pos)
    d = np.linalg.norm(pos[:, None] - pos[None], axis=-1)
    Jm = np.where((d < rc) & (d > 0), J, 0.0)
    axis = np.asarray(axis)
    muJ = mu * MUB

    def rhs(t, y):
        s = y.reshape(n, 3)
        H = Jm @ s + 2 * K * (s @ axis)[:, None] * axis[None]
        Bf = H / muJ + np.asarray(B)[None]
        c1 = np.cross(s, Bf)
        c2 = np.cross(s, c1)
        return (-GAMMA / (1 + alpha ** 2) * (c1 + alpha * c2)).reshape(-1)
    return rhs


def _cluster_case():
    pos = np.array([[0.0, 0, 0], [2.5, 0, 0], [1.25, 2.1, 0.3]])
    J = 3e-21
    init = np.array([_tilted(20, 0), _tilted(60, 100), _tilted(110, 230)])
    return pos, J, init


def _run_cluster(dt, tend, alpha, K, B):
    pos, J, init = _cluster_case()
    sysd = W.cluster(pos, J=J, rc=3.0, mu=2.0, B=B, T=0.0, alpha=alpha, dt=dt, K=K)
    o = O.Oracle(sysd)
    o.set_spins(init)
    o.step(int(round(tend / dt)))
    return o.spins()


def test_sweep_is_second_order_against_ode_reference():
    pos, J, init = _cluster_case()
    alpha, K, B = 0.1, 2e-22, (0.0, 3.0, 20.0)
    tend = 60 * FS
    rhs = _llg_rhs_factory(pos, J, 3.0, 2.0, K, [0, 0, 1], B, alpha)
    ref = solve_ivp(rhs, (0, tend), init.reshape(-1), method="DOP853", rtol=1e-13, atol=1e-15).y[:, -1]
    ref = ref.reshape(3, 3)
    errs = []
    for dt in (2.0 * FS, 1.0 * FS, 0.5 * FS):
        errs.append(np.abs(_run_cluster(dt, tend, alpha, K, B) - ref).max())
    o1 = np.log2(errs[0] / errs[1])
    o2 = np.log2(errs[1] / errs[2])
    assert 1.9 < o1 < 2.1 and 1.9 < o2 < 2.1, (errs, o1, o2)
    assert errs[-1] < 1e-4


def test_two_spin_exchange_precesses_about_total_spin():
    # two equal moments, alpha = 0, T = 0, no field: each spin rotates about
    # S = s1 + s2 at gamma J |S| / mu (an exact solution of Eq. 1)
    J, mu = 4e-21, 2.0
    pos = np.array([[0.0, 0, 0], [2.5, 0, 0]])
    s0 = np.array([_tilted(30, 0), _tilted(80, 140)])
    S = s0.sum(0)
    Sh = S / np.linalg.norm(S)
    w = GAMMA * J * np.linalg.norm(S) / (mu * MUB)
    tend = 40 * FS

    def exact(v, ang):
        return v * np.cos(ang) + np.cross(Sh, v) * np.sin(ang) + Sh * (Sh @ v) * (1 - np.cos(ang))

    want = np.array([exact(s0[0], w * tend), exact(s0[1], w * tend)])
    errs = []
    for dt in (0.4 * FS, 0.2 * FS):
        sysd = W.cluster(pos, J=J, rc=3.0, mu=mu, T=0.0, alpha=0.0, dt=dt)
        o = O.Oracle(sysd)
        o.set_spins(s0)
        o.step(int(round(tend / dt)))
        s = o.spins()
        errs.append(np.abs(s - want).max())
        # total spin and the pair energy are invariants of the exact flow and of
        # every sub-step of the sweep here
        assert np.allclose(s.sum(0), S, atol=5e-4)
        assert abs(s[0] @ s[1] - s0[0] @ s0[1]) < 1e-13
    assert 1.8 < np.log2(errs[0] / errs[1]) < 2.2
    assert errs[1] < 2e-3


def test_energy_conserved_to_rounding_without_damping():
    # alpha = 0, T = 0, exchange + Zeeman: each sub-step rotates s_i about a field
    # that does not depend on s_i, so every sub-step conserves the energy exactly
    sysd = W.bcc_fe(4, T=0.0, alpha=0.0, steps_dt=0.5 * FS, B=2.0)
    sysd["K"] = [0.0]
    o = O.Oracle(sysd)
    rng = np.random.default_rng(11)
    s = rng.normal(size=(o.n, 3))
    s /= np.linalg.norm(s, axis=1, keepdims=True)
    o.set_spins(s)
    e0 = o.observe()[10:13].sum()
    for _ in range(10):
        o.step(200)
        e = o.observe()[10:13].sum()
        assert abs(e - e0) <= 1e-12 * abs(e0)


def _aniso_energy_dev(dt, nsteps):
    sysd = W.bcc_fe(4, T=0.0, alpha=0.0, steps_dt=dt, B=2.0)
    sysd["K"] = [5e-3 * 1.602176634e-19]     # 100x the physical K, to make the error visible
    o = O.Oracle(sysd)
    rng = np.random.default_rng(12)
    s = rng.normal(size=(o.n, 3))
    s /= np.linalg.norm(s, axis=1, keepdims=True)
    o.set_spins(s)
    e0 = o.observe()[10:13].sum()
    dev = []
    for _ in range(10):
        o.step(nsteps // 10)
        dev.append(o.observe()[10:13].sum() - e0)
    return np.abs(dev).max() / abs(e0)


def test_energy_error_with_anisotropy_is_second_order():
    # with K != 0 the self-field depends on s_i, so sub-steps no longer conserve
    # the energy exactly; the error over a fixed time must fall as dt^2
    d1 = _aniso_energy_dev(1.0 * FS, 500)
    d2 = _aniso_energy_dev(0.5 * FS, 1000)
    assert d1 < 1e-3
    assert d1 / d2 > 3.3, (d1, d2)          # at least second order


def test_unit_norm_is_kept_every_step():
    sysd, ttm = W.config_gdfeco_32()
    sysd = W.gdfeco_sc(8)
    o = O.Oracle(sysd, W.ttm_single_cell(1500.0, 20 * FS))
    for _ in range(20):
        o.step(5)
        assert np.abs(np.linalg.norm(o.spins(), axis=1) - 1).max() <= 1e-14


def test_resume_by_stepcount_reproduces_trajectory():
    sysd = W.gdfeco_sc(6)
    a = O.Oracle(sysd)
    a.step(30)
    mid = a.spins()
    a.step(20)
    b = O.Oracle(sysd)
    b.set_spins(mid)
    b.stepcount = 30
    b.step(20)
    assert np.array_equal(a.spins(), b.spins())
