"""Seeded synthetic workloads, as plain dictionaries.

This module holds inputs only: system descriptions (lattice, species,
parameters, seeds) and TTM-grid descriptions, in the units of the C-ABI (SI,
moments in Bohr magnetons, lengths in angstrom).  It contains none of the
method's arithmetic and imports neither the CUDA binding nor the oracle, so
both sides can be fed from the same dictionaries.

Parameter sources: Table I and Sec. II.D of the paper (GdFeCo, moments,
damping, anisotropy), Sec. III.A (bcc Fe a = 2.8665 A, single-species
validation) and Sec. II.E (Bethe-Slater shape parameters of the bcc-Fe example
set, J2 = 0.2171, J3 = 1.841 A).
"""
import numpy as np

EV = 1.602176634e-19  # J per eV (input conversion only)
FS = 1e-15

# Bethe-Slater amplitude of the bcc-Fe example set (J2, J3 are the values the
# paper's Sec. II.E "66 % of nominal J1" figure pins).
FE_J1_EV = 0.02726
FE_J2 = 0.2171
FE_J3 = 1.841

ZERO_EXCH = {"kind": "none"}


def _exch2(ff, gg, fg):
    return [[ff, fg], [fg, gg]]


def bcc_fe(n=10, T=300.0, steps_dt=0.1 * FS, seed=42, B=1.0, alpha=0.1, sample_every=0):
    """Rigid bcc Fe, n^3 conventional cells, Bethe-Slater NN+NNN exchange
    (cutoff 3.5 A), uniaxial K = 5e-5 eV along z, field B along z."""
    bs = {"kind": "bethe_slater", "J1": FE_J1_EV * EV, "J2": FE_J2, "J3": FE_J3, "rc": 3.5}
    return {
        "lattice": "bcc", "nx": n, "ny": n, "nz": n, "a": 2.8665,
        "nspecies": 1, "mu": [2.2], "frac1": 0.0,
        "exch": [[bs]], "K": [5e-5 * EV], "axis": [0.0, 0.0, 1.0], "B": [0.0, 0.0, B],
        "alpha": [alpha], "dt": steps_dt, "T_bath": T,
        "init_dir": [[0.0, 0.0, 1.0]], "seed": seed, "sample_every": sample_every,
    }


def gdfeco_sc(n=32, seed=42, frac_gd=0.25, alpha=0.01, dt=0.1 * FS, T=300.0, B=0.0,
              sample_every=0):
    """Rigid GdFeCo on a simple-cubic lattice (a = 3.52 A), random Gd placement,
    constant nearest-neighbour exchange, Fe up / Gd down."""
    rc = 4.0  # between the first (3.52 A) and second (4.98 A) shells
    ff = {"kind": "const", "J1": 2.835e-21, "rc": rc}
    gg = {"kind": "const", "J1": 1.26e-21, "rc": rc}
    fg = {"kind": "const", "J1": -1.09e-21, "rc": rc}
    return {
        "lattice": "sc", "nx": n, "ny": n, "nz": n, "a": 3.52,
        "nspecies": 2, "mu": [1.92, 7.63], "frac1": frac_gd,
        "exch": _exch2(ff, gg, fg), "K": [8.07e-24, 8.07e-24], "axis": [0.0, 0.0, 1.0],
        "B": [0.0, 0.0, B], "alpha": [alpha, alpha], "dt": dt, "T_bath": T,
        "init_dir": [[0.0, 0.0, 1.0], [0.0, 0.0, -1.0]], "seed": seed,
        "sample_every": sample_every,
    }


def ttm_single_cell(peak_Te=1500.0, fwhm=50 * FS):
    """Homogeneous two-temperature model on one cell with a Gaussian pulse."""
    return {"cells": [1, 1, 1], "gamma_e": 225.0, "C_l": 3.1e6, "G": 1.7e18, "kappa_e": 0.0,
            "T0": 300.0, "source": "peak", "peak_Te": peak_Te, "fwhm": fwhm,
            "spatial": "uniform"}


def ttm_xy_spot(cells=16, peak_Te=2000.0, fwhm=50 * FS, sigma_xy=40.0, kappa_e=91.0):
    """Spatially resolved TTM grid with a Gaussian laser spot in the x-y plane."""
    return {"cells": [cells, cells, cells], "gamma_e": 225.0, "C_l": 3.1e6, "G": 1.7e18,
            "kappa_e": kappa_e, "T0": 300.0, "source": "peak", "peak_Te": peak_Te,
            "fwhm": fwhm, "spatial": "xy_gauss", "sigma_xy": sigma_xy}


def config_bcc_fe_2000():
    """bcc Fe 10x10x10 cells (2000 spins), 300 K, FP64 reference workload."""
    return bcc_fe(10)


def config_gdfeco_32():
    """GdFeCo sc 32^3 (32768 spins), one-cell 2TM, 50 fs pulse to 1500 K."""
    return gdfeco_sc(32), ttm_single_cell(1500.0, 50 * FS)


def config_gdfeco_large(n=128, realisations=4):
    """GdFeCo sc n^3 x realisations with a 16^3 TTM grid and a Gaussian spot."""
    s = gdfeco_sc(n)
    s["instances"] = [{"nx": n, "ny": n, "nz": n, "frac1": 0.25} for _ in range(realisations)]
    return s, ttm_xy_spot(16, 2000.0, 50 * FS)


def config_ensemble(n_peak=8, n_dur=8, n_real=16, seed=42, size_seed=7, lmin=12, lmax=24):
    """Batched phase-diagram ensemble: peak T_e x pulse duration x realisations
    of the GdFeCo model, each instance with its own cubic size and Gd fraction
    drawn from a seeded generator (inputs, not part of the method)."""
    rng = np.random.Generator(np.random.PCG64(size_seed))
    peaks = np.linspace(1000.0, 3000.0, n_peak)
    durs = np.linspace(25.0, 500.0, n_dur) * FS
    inst = []
    for iT in range(n_peak):
        for iD in range(n_dur):
            for r in range(n_real):
                L = int(rng.integers(lmin, lmax + 1))
                x = float(rng.uniform(0.20, 0.30))
                inst.append({"nx": L, "ny": L, "nz": L, "frac1": x,
                             "peak_Te": float(peaks[iT]), "fwhm": float(durs[iD])})
    s = gdfeco_sc(lmax, seed=seed)
    s["instances"] = inst
    return s, ttm_single_cell(1500.0, 50 * FS)


def single_spins(n, mu=1.92, B=(0.0, 0.0, 10.0), T=10.0, alpha=0.1, dt=1.0 * FS, K=0.0,
                 init=(0.0, 0.0, 1.0), seed=1234, nspecies=1, mu2=7.63, frac1=0.0):
    """n independent spins (sc lattice with no exchange), for single-spin laws."""
    return {
        "lattice": "sc", "nx": n, "ny": 1, "nz": 1, "a": 3.0,
        "nspecies": nspecies, "mu": [mu, mu2][:nspecies], "frac1": frac1,
        "exch": [[ZERO_EXCH] * nspecies for _ in range(nspecies)],
        "K": [K] * nspecies, "axis": [0.0, 0.0, 1.0], "B": list(B), "alpha": [alpha] * nspecies,
        "dt": dt, "T_bath": T, "init_dir": [list(init)] * nspecies, "seed": seed,
        "sample_every": 0,
    }


def cluster(positions, J, rc, mu=2.0, B=(0.0, 0.0, 0.0), T=0.0, alpha=0.0, dt=0.1 * FS,
            K=0.0, init=None, seed=99):
    """Open cluster of explicit positions with one constant exchange J (single
    species); init is a list of per-atom directions applied by the caller."""
    return {
        "lattice": "cluster", "positions": np.asarray(positions, dtype=np.float64),
        "species": np.zeros(len(positions), dtype=np.int32),
        "nspecies": 1, "mu": [mu], "frac1": 0.0,
        "exch": [[{"kind": "const", "J1": J, "rc": rc}]], "K": [K], "axis": [0.0, 0.0, 1.0],
        "B": list(B), "alpha": [alpha], "dt": dt, "T_bath": T,
        "init_dir": [list(init) if init is not None else [0.0, 0.0, 1.0]], "seed": seed,
        "sample_every": 0,
    }


AMU = 1.66053906660e-27
KB = 1.380649e-23


def morse_fe_lattice(spin_substeps=10, strain_amp=0.005, T_init=300.0, gamma_p=None, G=1.7e18, a=2.8665):
    """Moving-lattice block for bcc Fe: Morse pair potential (D = 0.4174 eV,
    alpha = 1.3885 1/A, r0 = 2.845 A, cutoff 5 A), 10 spin steps per lattice
    step, an initial sinusoidal strain along z and Maxwell-Boltzmann velocities.
    The electron-ion friction defaults to gamma_p = G m / (3 n_a k_B) with
    n_a = 2 / a^3 (the coefficient that reproduces a volumetric coupling G)."""
    m = 55.845 * AMU
    n_a = 2.0 / (a * 1e-10) ** 3
    if gamma_p is None:
        gamma_p = G * m / (3.0 * n_a * KB)
    return {"mass_amu": 55.845, "morse_D": 0.4174 * EV, "morse_alpha": 1.3885, "morse_r0": 2.845,
            "morse_rc": 5.0, "spin_substeps": spin_substeps, "strain_amp": strain_amp, "T_init": T_init,
            "gamma_p": gamma_p}


def ttm_z_exp(cells=(10, 10, 40), peak_Te=1500.0, fwhm=100 * FS, depth_frac=0.25, Lz=None, kappa_e=91.0):
    """TTM grid with a source decaying into the depth z (exp(-z / depth))."""
    return {"cells": list(cells), "gamma_e": 225.0, "C_l": 3.1e6, "G": 1.7e18, "kappa_e": kappa_e,
            "T0": 300.0, "source": "peak", "peak_Te": peak_Te, "fwhm": fwhm, "spatial": "z_exp",
            "depth_z": depth_frac * Lz}


def config_moving_fe(n=40):
    """Moving-lattice bcc Fe, n^3 cells, spin parameters of the bcc-Fe workload,
    Morse lattice, 1 fs lattice step with 10 spin sub-steps of 0.1 fs, TTM
    10x10x40 with a 100 fs pulse absorbed along z.  The electron heat
    capacity coefficient is 2250 J m^-3 K^-2 (ten times the GdFeCo value, as
    in the three-temperature workload): a 10 x 10 x 40 cell of this box holds
    about 32 atoms, and with 225 the electrons of a cell hold less energy than
    the ions exchange with them in one lattice step, so their energy goes
    negative within a step."""
    s = bcc_fe(n)
    lat = morse_fe_lattice()
    ttm = dict(ttm_z_exp((10, 10, 40), 1500.0, 100 * FS, 0.25, Lz=n * 2.8665), gamma_e=2250.0)
    return s, ttm, lat


def curie_scan(temps, n=6, reps=2, alpha=0.5, dt=1.0 * FS, seed=42):
    """Batched temperature scan of rigid bcc Fe (one uniform bath per
    instance): len(temps) x reps instances of n^3 cells, instance k at
    temps[k // reps]."""
    s = bcc_fe(n, T=float(temps[0]), steps_dt=dt, seed=seed, alpha=alpha)
    s["instances"] = [{"nx": n, "ny": n, "nz": n, "frac1": 0.0, "T_bath": float(T)}
                      for T in temps for _ in range(reps)]
    return s


# GdFeCo on fcc (Sec. II.D, Table I; shape re-derived as in Sec. II.E): literature amplitudes J1 per species
# pair, the radial shape re-derived for the fcc nearest-neighbour distance
# a / sqrt(2) (J2 = 0.4050, J3 = 3.1677 A), cutoff 3.4 A between the first two
# shells, K = 5.0384e-5 eV, alpha = 0.01, no field.
FCC_J2 = 0.4050
FCC_J3 = 3.1677


def gdfeco_fcc(n=13, seed=42, frac_gd=0.25, alpha=0.01, dt=0.2 * FS, T=300.0, sample_every=0):
    """Rigid fcc GdFeCo, n^3 conventional cells (4 n^3 atoms; n = 13 gives the
    paper's 8788), Fe up / Gd down."""
    def bs(j1_ev):
        return {"kind": "bethe_slater", "J1": j1_ev * EV, "J2": FCC_J2, "J3": FCC_J3, "rc": 3.4}
    return {
        "lattice": "fcc", "nx": n, "ny": n, "nz": n, "a": 3.6,
        "nspecies": 2, "mu": [1.92, 7.63], "frac1": frac_gd,
        "exch": _exch2(bs(0.01762), bs(0.007864), bs(-0.006803)),
        "K": [5.0384e-5 * EV, 5.0384e-5 * EV], "axis": [0.0, 0.0, 1.0], "B": [0.0, 0.0, 0.0],
        "alpha": [alpha, alpha], "dt": dt, "T_bath": T,
        "init_dir": [[0.0, 0.0, 1.0], [0.0, 0.0, -1.0]], "seed": seed, "sample_every": sample_every,
    }


def switching_campaign(peaks, ds, reps, n=13, t_peak=500 * FS, t_cool=500 * FS, t_tail=2000 * FS,
                       dt=0.2 * FS, sample_every=50, seed=42):
    """Peak T_e x cooling multiplier d x realisations of fcc GdFeCo under the
    three-stage step profile (peak for t_peak, half the peak for d t_cool,
    then 300 K).  Returns (system, bath, steps to the end of the longest
    run).  The stage base durations are inputs (the paper's are in its
    supplement, not available)."""
    s = gdfeco_fcc(n, seed=seed, dt=dt, sample_every=sample_every)
    s["instances"] = [{"nx": n, "ny": n, "nz": n, "frac1": 0.25, "peak_Te": float(T), "fwhm": float(d) * t_cool}
                      for T in peaks for d in ds for _ in range(reps)]
    bath = {"cells": [1, 1, 1], "gamma_e": 225.0, "C_l": 3.1e6, "G": 0.0, "kappa_e": 0.0, "T0": 300.0,
            "source": "step_profile", "peak_Te": float(peaks[0]), "fwhm": float(ds[0]) * t_cool, "t0": t_peak,
            "spatial": "uniform"}
    steps = int(round((t_peak + max(ds) * t_cool + t_tail) / dt))
    return s, bath, steps


def three_temperature(n=10, gamma_scale=1.0, sample_every=25):
    """Three-temperature relaxation of moving-lattice bcc Fe (paper Sec. III):
    electrons set to a hot T_e by the caller (tts_set_ttm_state) on one
    uniform cell without a source, lattice and spins starting at 300 K /
    aligned; gamma_scale multiplies the electron-ion friction."""
    s = bcc_fe(n, T=300.0, alpha=0.1, sample_every=sample_every)
    lat = morse_fe_lattice(strain_amp=0.0, T_init=300.0)
    lat["gamma_p"] *= gamma_scale
    # the lattice warms to ~400-550 K: atoms may stray 0.7 A from their sites, and
    # no two atoms within 3.5 + 1.4 A share a colour, so that no exchange pair
    # (3.5 A) can form inside one colour class as they move
    lat["skin"] = 1.4
    s["colour_rc"] = 4.9
    # gamma_e ten times the GdFeCo value: a one-cell electron reservoir then
    # holds enough energy that the ions' stochastic kicks never drive it
    # below zero (with 225 the reservoir of a 2000-atom box empties)
    bath = {"cells": [1, 1, 1], "gamma_e": 2250.0, "C_l": 3.1e6, "G": 1.7e18, "kappa_e": 0.0, "T0": 300.0,
            "source": "none", "spatial": "uniform"}
    return s, bath, lat
