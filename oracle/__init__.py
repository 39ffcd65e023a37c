"""ctypes view of the plain FP64 CPU oracle (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this package.  It never touches the CUDA library.

The system and TTM descriptions are the same plain dictionaries that the
input generators in ``paper_2608_18541_b300.workloads`` produce; this module
only copies them into the oracle's own C structs.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

NOBS = 20
_LIB = None


class _Exch(C.Structure):
    _fields_ = [("kind", C.c_int), ("J1", C.c_double), ("J2", C.c_double),
                ("J3", C.c_double), ("rc", C.c_double)]


class _Params(C.Structure):
    _fields_ = [
        ("lattice", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("a", C.c_double), ("n_explicit", C.c_int),
        ("pos_explicit", C.POINTER(C.c_double)), ("species_explicit", C.POINTER(C.c_int)),
        ("nspecies", C.c_int), ("mu", C.c_double * 2), ("frac1", C.c_double),
        ("exch", (_Exch * 2) * 2), ("K", C.c_double * 2), ("axis", C.c_double * 3),
        ("B", C.c_double * 3), ("alpha", C.c_double * 2), ("dt", C.c_double),
        ("T_bath", C.c_double), ("init_dir", (C.c_double * 3) * 2), ("seed", C.c_uint64),
        ("instance", C.c_uint32), ("sample_every", C.c_int), ("noise_mu_power", C.c_double),
        ("sweep", C.c_int), ("colour_rc", C.c_double),
    ]


class _Ttm(C.Structure):
    _fields_ = [
        ("ncx", C.c_int), ("ncy", C.c_int), ("ncz", C.c_int), ("gamma_e", C.c_double),
        ("C_l", C.c_double), ("G", C.c_double), ("kappa_e", C.c_double), ("T0", C.c_double),
        ("source", C.c_int), ("peak_Te", C.c_double), ("P0", C.c_double), ("fwhm", C.c_double),
        ("t0", C.c_double), ("spatial", C.c_int), ("sigma_xy", C.c_double), ("depth_z", C.c_double),
    ]


class _Lattice(C.Structure):
    _fields_ = [
        ("mass_amu", C.c_double), ("morse_D", C.c_double), ("morse_alpha", C.c_double),
        ("morse_r0", C.c_double), ("morse_rc", C.c_double), ("spin_substeps", C.c_int),
        ("strain_amp", C.c_double), ("T_init", C.c_double), ("gamma_p", C.c_double),
    ]


_LATTICE = {"sc": 0, "bcc": 1, "fcc": 2, "cluster": 3}
_EXKIND = {"none": 0, "const": 1, "bethe_slater": 2}
_SOURCE = {"none": 0, "peak": 1, "power": 2, "step_profile": 3}
_SPATIAL = {"uniform": 0, "xy_gauss": 1, "z_exp": 2}


def lib():
    global _LIB
    if _LIB is None:
        _LIB = _load(_build.build())
    return _LIB


def load_variant(path):
    """ctypes view of an altered oracle build (oracle.build.build_variant),
    for tests that show a pin fails on a planted mistake; pass it to Oracle
    as `library=`."""
    return _load(path)


def _load(path):
    L = C.CDLL(path)
    P = C.POINTER
    d, i64, u32 = C.c_double, C.c_int64, C.c_uint32
    L.orc_philox4x32_10.argtypes = [P(u32), P(u32), P(u32)]
    L.orc_uniform.argtypes = [u32]
    L.orc_uniform.restype = d
    L.orc_gauss3.argtypes = [P(u32), P(d)]
    L.orc_bethe_slater.argtypes = [d, d, d, d]
    L.orc_bethe_slater.restype = d
    L.orc_bethe_slater_deriv.argtypes = [d, d, d, d]
    L.orc_bethe_slater_deriv.restype = d
    L.orc_rederive_exchange.argtypes = [d, P(d), P(d), P(d)]
    L.orc_flow.argtypes = [P(d), P(d), d, d]
    L.orc_create.argtypes = [P(_Params), C.c_char_p, C.c_int]
    L.orc_create.restype = C.c_void_p
    L.orc_free.argtypes = [C.c_void_p]
    L.orc_set_ttm.argtypes = [C.c_void_p, P(_Ttm), C.c_char_p, C.c_int]
    L.orc_step.argtypes = [C.c_void_p, i64]
    for name in ("orc_natoms", "orc_ncolours", "orc_ttm_substeps", "orc_ttm_ncells"):
        getattr(L, name).argtypes = [C.c_void_p]
    L.orc_stepcount.argtypes = [C.c_void_p]
    L.orc_stepcount.restype = i64
    L.orc_set_stepcount.argtypes = [C.c_void_p, i64]
    L.orc_get_spins.argtypes = [C.c_void_p, P(d)]
    L.orc_set_spins.argtypes = [C.c_void_p, P(d)]
    L.orc_get_species.argtypes = [C.c_void_p, P(C.c_int)]
    L.orc_get_colours.argtypes = [C.c_void_p, P(C.c_int)]
    L.orc_get_positions.argtypes = [C.c_void_p, P(d)]
    L.orc_neighbour_count.argtypes = [C.c_void_p, C.c_int]
    L.orc_get_neighbours.argtypes = [C.c_void_p, C.c_int, P(C.c_int), P(d)]
    L.orc_field.argtypes = [C.c_void_p, C.c_int, P(d)]
    L.orc_observe.argtypes = [C.c_void_p, P(d)]
    L.orc_nsamples.argtypes = [C.c_void_p]
    L.orc_nsamples.restype = i64
    L.orc_get_samples.argtypes = [C.c_void_p, P(d)]
    L.orc_ttm_P0.argtypes = [C.c_void_p]
    L.orc_ttm_P0.restype = d
    L.orc_ttm_get.argtypes = [C.c_void_p, P(d), P(d)]
    L.orc_ttm_set.argtypes = [C.c_void_p, P(d), P(d)]
    L.orc_ttm_source_energy.argtypes = [C.c_void_p]
    L.orc_ttm_source_energy.restype = d
    L.orc_atom_cell.argtypes = [C.c_void_p, C.c_int]
    L.orc_set_lattice.argtypes = [C.c_void_p, P(_Lattice), C.c_char_p, C.c_int]
    L.orc_lattice_step.argtypes = [C.c_void_p, i64]
    L.orc_lattice_stepcount.argtypes = [C.c_void_p]
    L.orc_lattice_stepcount.restype = i64
    for name in ("orc_get_velocities", "orc_set_positions", "orc_set_velocities", "orc_get_forces"):
        getattr(L, name).argtypes = [C.c_void_p, P(d)]
    L.orc_lattice_energy.argtypes = [C.c_void_p, P(d), P(d)]
    L.orc_colour_violations.argtypes = [C.c_void_p]
    L.orc_ion_energy_to_electrons.argtypes = [C.c_void_p]
    L.orc_ion_energy_to_electrons.restype = d
    return L


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _iptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


# ---------------------------------------------------------------------------
# stateless helpers
# ---------------------------------------------------------------------------
def philox(ctr, key):
    L = lib()
    c = (C.c_uint32 * 4)(*[int(x) & 0xffffffff for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xffffffff for x in key])
    o = (C.c_uint32 * 4)()
    L.orc_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def uniform(x):
    return lib().orc_uniform(int(x) & 0xffffffff)


def gauss3(words):
    w = (C.c_uint32 * 4)(*[int(x) & 0xffffffff for x in words])
    g = (C.c_double * 3)()
    lib().orc_gauss3(w, g)
    return [g[0], g[1], g[2]]


def bethe_slater(r, J1, J2, J3):
    return lib().orc_bethe_slater(r, J1, J2, J3)


def bethe_slater_deriv(r, J1, J2, J3):
    return lib().orc_bethe_slater_deriv(r, J1, J2, J3)


def rederive_exchange(r1):
    x1, J2, J3 = C.c_double(), C.c_double(), C.c_double()
    rc = lib().orc_rederive_exchange(r1, C.byref(x1), C.byref(J2), C.byref(J3))
    if rc != 0:
        raise ValueError("no root")
    return x1.value, J2.value, J3.value


def flow(s, B, alpha, h):
    """One exact frozen-field sub-step of a single spin (in place on a copy)."""
    sv = np.ascontiguousarray(s, dtype=np.float64).copy()
    Bv = np.ascontiguousarray(B, dtype=np.float64)
    lib().orc_flow(_dptr(sv), _dptr(Bv), float(alpha), float(h))
    return sv


# ---------------------------------------------------------------------------
# system
# ---------------------------------------------------------------------------
def _fill_params(sysd, instance, index, noise_mu_power):
    p = _Params()
    inst = sysd.get("instances")
    over = inst[index] if inst else {}
    p.lattice = _LATTICE[sysd["lattice"]]
    p.nx = int(over.get("nx", sysd.get("nx", 1)))
    p.ny = int(over.get("ny", sysd.get("ny", 1)))
    p.nz = int(over.get("nz", sysd.get("nz", 1)))
    p.a = float(sysd.get("a", 1.0))
    keep = []
    if sysd["lattice"] == "cluster":
        pos = np.ascontiguousarray(sysd["positions"], dtype=np.float64).reshape(-1)
        spc = np.ascontiguousarray(sysd.get("species", np.zeros(pos.size // 3)), dtype=np.int32)
        keep += [pos, spc]
        p.n_explicit = pos.size // 3
        p.pos_explicit = _dptr(pos)
        p.species_explicit = _iptr(spc)
    ns = int(sysd["nspecies"])
    p.nspecies = ns
    for t in range(ns):
        p.mu[t] = float(sysd["mu"][t])
        p.K[t] = float(sysd["K"][t])
        p.alpha[t] = float(sysd["alpha"][t])
        d = sysd["init_dir"][t]
        for k in range(3):
            p.init_dir[t][k] = float(d[k])
    p.frac1 = float(over.get("frac1", sysd.get("frac1", 0.0)))
    for a in range(ns):
        for b in range(ns):
            e = sysd["exch"][a][b]
            x = p.exch[a][b]
            x.kind = _EXKIND[e["kind"]]
            x.J1 = float(e.get("J1", 0.0))
            x.J2 = float(e.get("J2", 0.0))
            x.J3 = float(e.get("J3", 1.0))
            x.rc = float(e.get("rc", 0.0))
    for k in range(3):
        p.axis[k] = float(sysd["axis"][k])
        p.B[k] = float(sysd["B"][k])
    p.dt = float(sysd["dt"])
    p.T_bath = float(over.get("T_bath", sysd.get("T_bath", 0.0)))
    p.seed = int(sysd["seed"])
    p.instance = int(instance)
    p.sample_every = int(sysd.get("sample_every", 0))
    p.noise_mu_power = float(noise_mu_power)
    p.sweep = {"symmetric": 0, "merged": 1}[sysd.get("sweep", "symmetric")]
    p.colour_rc = float(sysd.get("colour_rc", 0.0))
    return p, keep


def _fill_ttm(t, over):
    x = _Ttm()
    x.ncx, x.ncy, x.ncz = (int(v) for v in t["cells"])
    x.gamma_e = float(t["gamma_e"])
    x.C_l = float(t["C_l"])
    x.G = float(t["G"])
    x.kappa_e = float(t.get("kappa_e", 0.0))
    x.T0 = float(t["T0"])
    x.source = _SOURCE[t.get("source", "none")]
    x.peak_Te = float(over.get("peak_Te", t.get("peak_Te", 0.0)))
    x.P0 = float(t.get("P0", 0.0))
    x.fwhm = float(over.get("fwhm", t.get("fwhm", 1e-13)))
    x.t0 = float(t.get("t0", -1.0))
    x.spatial = _SPATIAL[t.get("spatial", "uniform")]
    x.sigma_xy = float(t.get("sigma_xy", 1.0))
    x.depth_z = float(t.get("depth_z", 1.0))
    return x


class Oracle:
    """One instance (realisation) of a system description, advanced on the CPU.

    instance: the realisation id that keys the noise and the alloy placement;
    index: the entry of sysd["instances"] that gives its size, composition and
    pulse (defaults to `instance`)."""

    def __init__(self, sysd, ttm=None, instance=0, noise_mu_power=0.5, index=None, lattice=None,
                 library=None):
        self._L = L = library if library is not None else lib()
        index = instance if index is None else index
        p, self._keep = _fill_params(sysd, instance, index, noise_mu_power)
        err = C.create_string_buffer(256)
        h = L.orc_create(C.byref(p), err, 256)
        if not h:
            raise ValueError(err.value.decode())
        self._h = h
        self.n = L.orc_natoms(h)
        if lattice is not None:
            x = _Lattice()
            for name, _ in _Lattice._fields_:
                setattr(x, name, lattice[name])
            if L.orc_set_lattice(h, C.byref(x), err, 256) != 0:
                raise ValueError(err.value.decode())
        if ttm is not None:
            inst = sysd.get("instances")
            over = inst[index] if inst else {}
            t = _fill_ttm(ttm, over)
            if L.orc_set_ttm(h, C.byref(t), err, 256) != 0:
                raise ValueError(err.value.decode())

    def __del__(self):
        if getattr(self, "_h", None) and getattr(self, "_L", None) is not None:
            self._L.orc_free(self._h)
            self._h = None

    def step(self, n):
        self._L.orc_step(self._h, int(n))

    @property
    def ncolours(self):
        return self._L.orc_ncolours(self._h)

    @property
    def stepcount(self):
        return self._L.orc_stepcount(self._h)

    @stepcount.setter
    def stepcount(self, n):
        self._L.orc_set_stepcount(self._h, int(n))

    def spins(self):
        out = np.empty((self.n, 3), dtype=np.float64)
        self._L.orc_get_spins(self._h, _dptr(out))
        return out

    def set_spins(self, s):
        s = np.ascontiguousarray(s, dtype=np.float64).reshape(self.n, 3)
        self._L.orc_set_spins(self._h, _dptr(s))

    def species(self):
        out = np.empty(self.n, dtype=np.int32)
        self._L.orc_get_species(self._h, _iptr(out))
        return out

    def colours(self):
        out = np.empty(self.n, dtype=np.int32)
        self._L.orc_get_colours(self._h, _iptr(out))
        return out

    def positions(self):
        out = np.empty((self.n, 3), dtype=np.float64)
        self._L.orc_get_positions(self._h, _dptr(out))
        return out

    def neighbours(self, i):
        L = self._L
        m = L.orc_neighbour_count(self._h, int(i))
        j = np.empty(m, dtype=np.int32)
        J = np.empty(m, dtype=np.float64)
        L.orc_get_neighbours(self._h, int(i), _iptr(j), _dptr(J))
        return j, J

    def field(self, i):
        out = np.empty(3, dtype=np.float64)
        self._L.orc_field(self._h, int(i), _dptr(out))
        return out

    def observe(self):
        out = np.empty(NOBS, dtype=np.float64)
        self._L.orc_observe(self._h, _dptr(out))
        return out

    def samples(self):
        L = self._L
        m = L.orc_nsamples(self._h)
        out = np.empty((m, NOBS), dtype=np.float64)
        if m:
            L.orc_get_samples(self._h, _dptr(out))
        return out

    @property
    def P0(self):
        return self._L.orc_ttm_P0(self._h)

    @property
    def ttm_substeps(self):
        return self._L.orc_ttm_substeps(self._h)

    def ttm(self):
        L = self._L
        nc = L.orc_ttm_ncells(self._h)
        Te = np.empty(nc)
        Tl = np.empty(nc)
        if nc:
            L.orc_ttm_get(self._h, _dptr(Te), _dptr(Tl))
        return Te, Tl

    def set_ttm_state(self, Te, Tl):
        Te = np.ascontiguousarray(Te, dtype=np.float64)
        Tl = np.ascontiguousarray(Tl, dtype=np.float64)
        self._L.orc_ttm_set(self._h, _dptr(Te), _dptr(Tl))

    @property
    def source_energy(self):
        return self._L.orc_ttm_source_energy(self._h)

    def atom_cell(self, i):
        return self._L.orc_atom_cell(self._h, int(i))

    # -- moving lattice -------------------------------------------------------
    def lattice_step(self, n):
        self._L.orc_lattice_step(self._h, int(n))

    @property
    def lattice_stepcount(self):
        return self._L.orc_lattice_stepcount(self._h)

    def velocities(self):
        out = np.empty((self.n, 3))
        self._L.orc_get_velocities(self._h, _dptr(out))
        return out

    def set_velocities(self, v):
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(self.n, 3)
        self._L.orc_set_velocities(self._h, _dptr(v))

    def set_positions(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(self.n, 3)
        self._L.orc_set_positions(self._h, _dptr(x))

    def forces(self):
        out = np.empty((self.n, 3))
        self._L.orc_get_forces(self._h, _dptr(out))
        return out

    def lattice_energy(self):
        k, m = C.c_double(), C.c_double()
        self._L.orc_lattice_energy(self._h, C.byref(k), C.byref(m))
        return k.value, m.value

    def total_energy(self):
        k, m = self.lattice_energy()
        o = self.observe()
        return k + m + o[10] + o[11] + o[12]

    @property
    def colour_violations(self):
        return self._L.orc_colour_violations(self._h)

    @property
    def ion_energy_to_electrons(self):
        return self._L.orc_ion_energy_to_electrons(self._h)
