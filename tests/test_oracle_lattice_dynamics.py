"""Oracle pins for the moving lattice (paper Sec. II.A: positions evolve under
the pair potential plus the exchange-mediated force -dJ/dr (s_i.s_j), spins
and lattice advanced together by a symmetric splitting).

Checks: forces are minus the gradient of an energy computed independently;
total momentum is conserved; without damping or noise the total energy error
is bounded and falls as dt^2; the electron-ion Ornstein-Uhlenbeck coupling
brings the ions to the bath temperature; with a TTM grid the energy handed to
the electrons plus the source balances the total energy.
"""
import numpy as np

import oracle as O
from paper_2608_18541_b300 import workloads as W

FS = 1e-15
EV = 1.602176634e-19
KB = 1.380649e-23


def _quiet_fe(n=5, K=0.0, B=0.5):
    s = W.bcc_fe(n, T=0.0, alpha=0.0, B=B)
    s["K"] = [K]
    return s


def _energy_independent(o, sysd, lat, pos, spins):
    """Morse + Bethe-Slater exchange + Zeeman + anisotropy, all pairs by
    brute force with the minimum image (independent of the oracle's lists)."""
    n = len(pos)
    box = np.array([sysd["nx"], sysd["ny"], sysd["nz"]]) * sysd["a"]
    d = pos[None, :, :] - pos[:, None, :]
    d -= box * np.round(d / box)
    r = np.sqrt((d ** 2).sum(-1)) + np.eye(n)
    D, al, r0, rc = lat["morse_D"], lat["morse_alpha"], lat["morse_r0"], lat["morse_rc"]

    def U(x):
        e = np.exp(-al * (x - r0))
        return D * (e * e - 2 * e)

    def dU(x):
        e = np.exp(-al * (x - r0))
        return 2 * al * D * (e - e * e)

    # shifted-force Morse: energy and force vanish at the cutoff
    mask = (r < rc) & ~np.eye(n, dtype=bool)
    em = 0.5 * np.where(mask, U(r) - U(rc) - (r - rc) * dU(rc), 0.0).sum()
    e = sysd["exch"][0][0]
    x = (r / e["J3"]) ** 2
    J = np.where((r < e["rc"]) & ~np.eye(n, dtype=bool), 4 * e["J1"] * x * (1 - e["J2"] * x) * np.exp(-x), 0.0)
    eex = -0.5 * np.einsum("ij,ik,jk->", J, spins, spins)
    mu = sysd["mu"][0] * 9.2740100783e-24
    ez = -(mu * spins @ np.array(sysd["B"])).sum()
    ean = -(sysd["K"][0] * (spins @ np.array(sysd["axis"])) ** 2).sum()
    return em + eex + ez + ean


def test_forces_are_minus_energy_gradient():
    sysd = _quiet_fe(4, K=1e-22)
    lat = W.morse_fe_lattice(T_init=300.0, gamma_p=0.0, strain_amp=0.02)
    o = O.Oracle(sysd, None, lattice=lat)
    rng = np.random.default_rng(4)
    s = rng.normal(size=(o.n, 3))
    s /= np.linalg.norm(s, axis=1, keepdims=True)
    o.set_spins(s)
    pos = o.positions() + rng.normal(scale=0.05, size=(o.n, 3))
    pos[0] = pos[1] + np.array([4.995, 0.0, 0.0])   # one pair right at the Morse cutoff
    o.set_positions(pos)
    pos = o.positions()
    F = o.forces()
    h = 1e-5
    for i in (0, 7, 30):
        for k in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, k] += h
            pm[i, k] -= h
            g = (_energy_independent(o, sysd, lat, pp, s) - _energy_independent(o, sysd, lat, pm, s)) / (2 * h * 1e-10)
            assert abs(F[i, k] + g) < 1e-6 * np.abs(F).max(), (i, k, F[i, k], -g)
    # the oracle's own energies agree with the independent sum
    k_e, m_e = o.lattice_energy()
    ob = o.observe()
    assert np.isclose(m_e + ob[10] + ob[11] + ob[12], _energy_independent(o, sysd, lat, pos, s), rtol=1e-11)


def test_momentum_conserved_and_colours_stay_valid():
    sysd = _quiet_fe(5)
    o = O.Oracle(sysd, None, lattice=W.morse_fe_lattice(T_init=600.0, gamma_p=0.0))
    M = 55.845 * W.AMU
    assert np.abs(M * o.velocities().sum(0)).max() < 1e-30
    o.lattice_step(50)
    p = M * o.velocities().sum(0)
    scale = M * np.abs(o.velocities()).sum()
    assert np.abs(p).max() < 1e-12 * scale
    assert o.colour_violations == 0


def _energy_error(dt_fs, nsteps):
    sysd = _quiet_fe(5)
    sysd["dt"] = dt_fs * FS / 10
    o = O.Oracle(sysd, None, lattice=W.morse_fe_lattice(T_init=300.0, gamma_p=0.0))
    rng = np.random.default_rng(9)
    s = np.array([0, 0, 1.0]) + rng.normal(scale=0.2, size=(o.n, 3))
    s /= np.linalg.norm(s, axis=1, keepdims=True)
    o.set_spins(s)
    e0 = o.total_energy()
    dev = 0.0
    for _ in range(10):
        o.lattice_step(nsteps // 10)
        dev = max(dev, abs(o.total_energy() - e0))
    kin = o.lattice_energy()[0]
    return dev / kin


def test_energy_error_bounded_and_second_order():
    d1 = _energy_error(1.0, 200)
    d2 = _energy_error(0.5, 400)
    assert d1 < 0.05                     # relative to the kinetic energy
    assert d1 / d2 > 3.3, (d1, d2)


def test_ornstein_uhlenbeck_coupling_thermalises_ions():
    sysd = _quiet_fe(5)
    sysd["T_bath"] = 500.0
    lat = W.morse_fe_lattice(T_init=100.0)
    lat["gamma_p"] *= 20.0                 # relaxation time M / gamma ~ 0.1 ps
    o = O.Oracle(sysd, None, lattice=lat)
    o.lattice_step(400)
    T = []
    for _ in range(40):
        o.lattice_step(10)
        T.append(2 * o.lattice_energy()[0] / (3 * o.n * KB))
    T = np.array(T)
    # equipartition with the potential energy half: kinetic temperature = bath
    assert abs(T.mean() - 500.0) < 0.04 * 500.0, T.mean()


def test_energy_balance_with_electrons_and_source():
    sysd = _quiet_fe(6)
    ttm = W.ttm_z_exp((2, 2, 4), 900.0, 40 * FS, 0.25, Lz=6 * 2.8665)
    lat = W.morse_fe_lattice(T_init=300.0)
    o = O.Oracle(sysd, ttm, lattice=lat)
    V = (6 * 2.8665e-10) ** 3 / 16

    def total():
        Te, _ = o.ttm()
        return o.total_energy() + (0.5 * ttm["gamma_e"] * Te ** 2).sum() * V

    e0 = total()
    o.lattice_step(150)
    dep = o.source_energy
    assert dep > 0
    err = abs(total() - e0 - dep)
    # what remains is the splitting error of the conservative part
    assert err < 0.02 * o.lattice_energy()[0], (err, dep)
