"""Oracle pins: the two-temperature-model grid (fix ttm of Sec. II.B) --
energy balance, an independent ODE integration, a diffusion eigenmode, the
peak calibration of the source and the atom-to-cell map of Eq. 2."""
import numpy as np
from scipy.integrate import solve_ivp

import oracle as O
from paper_2608_18541_b300 import workloads as W

FS = 1e-15


def _spot_grid(cells=4, n=8, kappa=91.0):
    sysd = W.gdfeco_sc(n, T=300.0)
    ttm = W.ttm_xy_spot(cells, 1200.0, 30 * FS, sigma_xy=8.0, kappa_e=kappa)
    return sysd, ttm


def test_energy_balance_is_exact():
    # sum over cells of (gamma_e Te^2 / 2 + C_l Tl) V changes only by the source
    sysd, ttm = _spot_grid()
    o = O.Oracle(sysd, ttm)
    assert o.ttm_substeps > 1
    V = (8 * 3.52e-10) ** 3 / 64

    def energy():
        Te, Tl = o.ttm()
        return ((0.5 * ttm["gamma_e"] * Te ** 2 + ttm["C_l"] * Tl) * V).sum()

    e0 = energy()
    for _ in range(6):
        o.step(200)
        dep = o.source_energy
        assert dep > 0
        assert abs(energy() - e0 - dep) < 1e-12 * dep


def test_single_cell_converges_to_ode_solution_at_first_order():
    # explicit sub-steps of the 2TM: error against an accurate ODE integration
    # of gamma_e Te dTe/dt = -G (Te - Tl) + S(t), C_l dTl/dt = G (Te - Tl)
    ttm = W.ttm_single_cell(1500.0, 50 * FS)
    tend = 300 * FS
    res = {}
    for dt in (0.2 * FS, 0.1 * FS):
        sysd = W.single_spins(1, T=0.0, dt=dt)
        o = O.Oracle(sysd, ttm)
        o.step(int(round(tend / dt)))
        res[dt] = (o.ttm(), o.P0)
    P0 = res[0.1 * FS][1]
    sig = ttm["fwhm"] / (2 * np.sqrt(2 * np.log(2)))
    t0 = 3 * sig

    def rhs(t, y):
        Te, Tl = y
        S = P0 * np.exp(-(t - t0) ** 2 / (2 * sig ** 2))
        return [(-ttm["G"] * (Te - Tl) + S) / (ttm["gamma_e"] * Te), ttm["G"] * (Te - Tl) / ttm["C_l"]]

    ref = solve_ivp(rhs, (0, tend), [300.0, 300.0], method="DOP853", rtol=1e-12, atol=1e-9).y[:, -1]
    # run both dt with the same P0 so only the time discretisation differs
    errs = []
    for dt in (0.2 * FS, 0.1 * FS):
        t2 = dict(ttm, source="power", P0=P0)
        o = O.Oracle(W.single_spins(1, T=0.0, dt=dt), t2)
        o.step(int(round(tend / dt)))
        Te, Tl = o.ttm()
        errs.append(max(abs(Te[0] - ref[0]), abs(Tl[0] - ref[1])))
    assert errs[1] < 1.0                       # kelvin
    assert 1.8 < errs[0] / errs[1] < 2.2       # explicit scheme: first order


def test_peak_calibration_hits_target():
    for peak, fwhm in ((1500.0, 50 * FS), (2600.0, 25 * FS)):
        ttm = W.ttm_single_cell(peak, fwhm)
        o = O.Oracle(W.single_spins(1, T=0.0, dt=0.1 * FS), ttm)
        mx = 0.0
        for _ in range(int(round((3 + 10) * fwhm / 2.3548 / (0.1 * FS)))):
            o.step(1)
            mx = max(mx, o.ttm()[0][0])
        assert abs(mx - peak) < 1e-9


def test_diffusion_eigenmode_decay():
    # no coupling, no source, a small cosine along x: the amplitude decays as
    # exp(-kappa lambda t / C_e) with lambda = (2 - 2 cos(2 pi / n)) / dx^2, the
    # eigenvalue of the periodic 7-point Laplacian
    n = 16
    sysd = W.single_spins(32, T=0.0, dt=0.1 * FS)      # box 32 x 3 A along x
    ttm = {"cells": [n, 1, 1], "gamma_e": 225.0, "C_l": 3.1e6, "G": 0.0, "kappa_e": 91.0,
           "T0": 300.0, "source": "none"}
    o = O.Oracle(sysd, ttm)
    x = (np.arange(n) + 0.5) / n
    eps = 1e-3
    Te0 = 300.0 + eps * np.cos(2 * np.pi * x)
    o.set_ttm_state(Te0, np.full(n, 300.0))
    steps = 3000
    o.step(steps)
    Te, _ = o.ttm()
    amp = 2 * (Te * np.cos(2 * np.pi * x)).mean()
    dx = 32 * 3.0e-10 / n
    lam = (2 - 2 * np.cos(2 * np.pi / n)) / dx ** 2
    t = steps * 0.1 * FS
    want = eps * np.exp(-91.0 * lam * t / (225.0 * 300.0))
    assert want < 0.9 * eps                              # a real decay happened
    assert abs(amp - want) < 2e-3 * (eps - want)


def test_atom_to_cell_map():
    # Eq. 2 reads T_e of the cell holding the atom: floor(x / L * n), and atoms
    # exactly on a cell face belong to the upper cell
    sysd = W.gdfeco_sc(12)
    for cells in ([4, 3, 2], [5, 7, 3]):
        ttm = {"cells": cells, "gamma_e": 225.0, "C_l": 3.1e6, "G": 1.7e18, "kappa_e": 0.0,
               "T0": 300.0, "source": "none"}
        o = O.Oracle(sysd, ttm)
        pos = o.positions()
        L = 12 * 3.52
        for i in range(0, o.n, 7):
            c = []
            for d in range(3):
                f = pos[i, d] / L * cells[d]
                k = int(np.floor(f + 1e-9))     # faces go up
                c.append(k)
            assert o.atom_cell(i) == (c[2] * cells[1] + c[1]) * cells[0] + c[0]
