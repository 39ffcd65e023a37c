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


# ---------------------------------------------------------------------------
# The laser source's spatial profile (Sec. II.B, fix ttm source term), pinned
# by integral identities rather than by its formula.  With no diffusion and
# no electron-phonon exchange each cell only collects its own source, so the
# electron energy gained per cell, gamma_e (Te^2 - T0^2) / 2, is proportional
# to the profile f at that cell's centre, and the deposits normalised to sum 1
# are f / sum(f) whatever the pulse and its time quadrature.
#  - xy Gaussian exp(-r^2 / (2 sigma^2)) sampled on a grid of spacing d much
#    finer than sigma and truncated far in its tail: by Poisson summation the
#    sampled sums equal the integrals up to exp(-2 pi^2 sigma^2 / d^2), so the
#    normalised deposits have mean the box centre and variance sigma^2 along
#    x and y, and sum(f) over one z layer is 2 pi sigma^2 / d^2; the deposit
#    of the centre cell of an odd grid (f = 1) is then d^2 / (2 pi sigma^2 nz).
#  - exp(-z / depth): adjacent z layers differ by exactly exp(-dz / depth),
#    and the whole profile carries sum_k exp(-(k + 1/2) dz / depth) per column,
#    a geometric series, relative to a uniform source of the same pulse.
# ---------------------------------------------------------------------------
import os
import tempfile

import pytest

from oracle import build as OB

_SPOT_N = 24            # sc cells per edge: box 84.48 A
_SPOT_SIGMA = 6.0       # angstrom: the box half-width is 7 sigma


def _deposits(ttm, library=None, n=_SPOT_N):
    """Per-cell source energy (relative) after the whole pulse, no diffusion,
    no e-ph exchange."""
    sysd = W.gdfeco_sc(n, T=0.0, dt=0.5 * FS)
    o = O.Oracle(sysd, ttm, library=library)
    o.step(24)                          # t0 + 10 sigma_t of a 2 fs pulse is < 12 fs
    Te, _ = o.ttm()
    d = Te ** 2 - ttm["T0"] ** 2
    return d, o.source_energy


def _spot_ttm(cells, spatial="xy_gauss", depth=None):
    t = {"cells": list(cells), "gamma_e": 225.0, "C_l": 3.1e6, "G": 0.0, "kappa_e": 0.0, "T0": 300.0,
         "source": "power", "P0": 1e21, "fwhm": 2 * FS, "spatial": spatial}
    if spatial == "xy_gauss":
        t["sigma_xy"] = _SPOT_SIGMA
    if spatial == "z_exp":
        t["depth_z"] = depth
    return t


def _spot_stats(dep, cells, box):
    nx, ny, nz = cells
    p = (dep / dep.sum()).reshape(nz, ny, nx)
    dx, dy = box / nx, box / ny
    x = (np.arange(nx) + 0.5) * dx - 0.5 * box
    y = (np.arange(ny) + 0.5) * dy - 0.5 * box
    px, py = p.sum(axis=(0, 1)), p.sum(axis=(0, 2))
    return p, (px * x).sum(), (py * y).sum(), (px * x * x).sum(), (py * y * y).sum(), dx, dy


@pytest.mark.parametrize("cells", [(21, 21, 2), (20, 20, 3), (21, 16, 1)])
def test_xy_gaussian_spot_moments_and_normalisation(cells):
    box = _SPOT_N * 3.52
    dep, _ = _deposits(_spot_ttm(cells))
    p, mx, my, vx, vy, dx, dy = _spot_stats(dep, cells, box)
    s2 = _SPOT_SIGMA ** 2
    assert abs(mx) < 1e-9 * box and abs(my) < 1e-9 * box         # centred on the box
    assert abs(vx / s2 - 1) < 1e-9 and abs(vy / s2 - 1) < 1e-9   # variance sigma^2: the 2 of 2 sigma^2
    # uniform through the depth
    for k in range(1, cells[2]):
        assert np.allclose(p[k], p[0], rtol=1e-12, atol=1e-300)
    if cells[0] % 2 and cells[1] % 2:
        # the centre cell holds f = 1: its share is d^2 / (2 pi sigma^2 nz)
        want = dx * dy / (2 * np.pi * s2 * cells[2])
        assert abs(p[0, cells[1] // 2, cells[0] // 2] / want - 1) < 1e-9


def test_z_exponential_profile_ratios_and_total():
    box = _SPOT_N * 3.52
    cells = (3, 2, 12)
    depth = 0.25 * box
    dep, e_exp = _deposits(_spot_ttm(cells, "z_exp", depth))
    dep = dep.reshape(cells[2], cells[1], cells[0])
    dz = box / cells[2]
    r = dep[1:] / dep[:-1]
    assert np.allclose(r, np.exp(-dz / depth), rtol=1e-12)       # decays into +z at 1/depth
    assert np.allclose(dep, dep[:, :1, :1], rtol=1e-12)            # uniform in x-y
    # total against a uniform source of the same pulse: the mean of f over the
    # grid is (1/nz) sum_k exp(-(k + 1/2) dz / depth), a geometric series
    _, e_uni = _deposits(_spot_ttm(cells, "uniform"))
    q = np.exp(-dz / depth)
    want = np.exp(-0.5 * dz / depth) * (1 - q ** cells[2]) / (1 - q) / cells[2]
    assert abs(e_exp / e_uni / want - 1) < 1e-12


@pytest.mark.parametrize("plant,spatial", [("ORC_PLANT_SPOT_NO_HALF", "xy_gauss"),
                                           ("ORC_PLANT_SPOT_OFF_CENTRE", "xy_gauss"),
                                           ("ORC_PLANT_DEPTH_SIGN", "z_exp")])
def test_source_pins_catch_planted_mistakes(plant, spatial):
    # an oracle built with one deliberate error in the profile fails the pins
    with tempfile.TemporaryDirectory() as tmp:
        bad = O.load_variant(OB.build_variant([plant], tmp))
        box = _SPOT_N * 3.52
        if spatial == "xy_gauss":
            cells = (21, 21, 2)
            dep, _ = _deposits(_spot_ttm(cells), library=bad)
            p, mx, my, vx, vy, dx, dy = _spot_stats(dep, cells, box)
            centred = abs(mx) < 1e-9 * box and abs(my) < 1e-9 * box
            width = abs(vx / _SPOT_SIGMA ** 2 - 1) < 1e-9 and abs(vy / _SPOT_SIGMA ** 2 - 1) < 1e-9
            peak = abs(p[0, 10, 10] / (dx * dy / (2 * np.pi * _SPOT_SIGMA ** 2 * 2)) - 1) < 1e-9
            assert not (centred and width and peak)
        else:
            cells = (3, 2, 12)
            depth = 0.25 * box
            dep, _ = _deposits(_spot_ttm(cells, "z_exp", depth), library=bad)
            dep = dep.reshape(cells[2], cells[1], cells[0])
            assert not np.allclose(dep[1:] / dep[:-1], np.exp(-(box / cells[2]) / depth), rtol=1e-12)
