"""Python binding of the tts C ABI (include/tts.h): argument marshalling only.

Every computation runs in the CUDA library ``libtts.so`` built in this
directory (``python -m paper_2608_18541_b300.build`` or
``__graft_entry__.build()``).  There is no fallback: if the library is
missing, loading fails with an error.

System and TTM descriptions are the plain dictionaries of
``paper_2608_18541_b300.workloads``.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtts.so")

TTS_OK = 0
ERRORS = {-1: "TTS_ERR_ARG", -2: "TTS_ERR_CUDA", -3: "TTS_ERR_OOM", -4: "TTS_ERR_DEVICE_TIMEOUT",
          -5: "TTS_ERR_HEALTH", -6: "TTS_ERR_STATE", -7: "TTS_ERR_UNSUPPORTED"}
NOBS = 20
MAX_SPECIES = 2

LATTICE = {"sc": 0, "bcc": 1, "fcc": 2, "cluster": 3}
EXCH = {"none": 0, "const": 1, "bethe_slater": 2}
ENGINE = {"auto": 0, "general": 1, "checker": 2, "resident": 3}
ENGINE_NAME = {v: k for k, v in ENGINE.items()}
SOURCE = {"none": 0, "peak": 1, "power": 2, "step_profile": 3}
SPATIAL = {"uniform": 0, "xy_gauss": 1, "z_exp": 2}


class TTSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (ERRORS.get(code, code), msg))
        self.code = code


class tts_exchange(C.Structure):
    _fields_ = [("kind", C.c_int), ("J1", C.c_double), ("J2", C.c_double), ("J3", C.c_double),
                ("rc", C.c_double)]


class tts_system_desc(C.Structure):
    _fields_ = [
        ("lattice", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("a", C.c_double),
        ("n_explicit", C.c_int), ("pos_explicit", C.POINTER(C.c_double)),
        ("species_explicit", C.POINTER(C.c_int)), ("nspecies", C.c_int),
        ("mu_muB", C.c_double * MAX_SPECIES), ("frac1", C.c_double),
        ("exch", (tts_exchange * MAX_SPECIES) * MAX_SPECIES), ("K", C.c_double * MAX_SPECIES),
        ("axis", C.c_double * 3), ("B", C.c_double * 3), ("alpha", C.c_double * MAX_SPECIES),
        ("dt", C.c_double), ("T_bath", C.c_double), ("init_dir", (C.c_double * 3) * MAX_SPECIES),
        ("seed", C.c_uint64), ("precision", C.c_int), ("sample_every", C.c_int),
        ("obs_capacity", C.c_int), ("n_instances", C.c_int), ("inst_cells", C.POINTER(C.c_int)),
        ("inst_frac1", C.POINTER(C.c_double)), ("inst_peak_Te", C.POINTER(C.c_double)),
        ("inst_fwhm", C.POINTER(C.c_double)), ("engine", C.c_int), ("instance_base", C.c_int),
        ("sweep", C.c_int), ("inst_T_bath", C.POINTER(C.c_double)), ("colour_rc", C.c_double),
    ]


class tts_ttm_desc(C.Structure):
    _fields_ = [
        ("cells", C.c_int * 3), ("gamma_e", C.c_double), ("C_l", C.c_double), ("G", C.c_double),
        ("kappa_e", C.c_double), ("T0", C.c_double), ("source", C.c_int), ("peak_Te", C.c_double),
        ("P0", C.c_double), ("fwhm", C.c_double), ("t0", C.c_double), ("spatial", C.c_int),
        ("sigma_xy", C.c_double), ("depth_z", C.c_double),
    ]


class tts_lattice_desc(C.Structure):
    _fields_ = [
        ("mass_amu", C.c_double), ("morse_D", C.c_double), ("morse_alpha", C.c_double),
        ("morse_r0", C.c_double), ("morse_rc", C.c_double), ("spin_substeps", C.c_int),
        ("strain_amp", C.c_double), ("T_init", C.c_double), ("gamma_p", C.c_double), ("skin", C.c_double),
    ]


class tts_info_t(C.Structure):
    _fields_ = [("n_total", C.c_int64), ("n_instances", C.c_int), ("engine", C.c_int),
                ("precision", C.c_int), ("max_colours", C.c_int), ("steps_done", C.c_int64),
                ("kernel_launches", C.c_int64)]


# (name, argtypes); every function returns int except tts_last_error
_P = C.POINTER
_SIG = {
    "tts_create_system": [_P(tts_system_desc), C.c_void_p, _P(C.c_void_p)],
    "tts_destroy": [C.c_void_p],
    "tts_set_ttm_grid": [C.c_void_p, _P(tts_ttm_desc)],
    "tts_step": [C.c_void_p, C.c_int64],
    "tts_sync": [C.c_void_p],
    "tts_observables": [C.c_void_p, C.c_int, _P(C.c_double), C.c_int64, _P(C.c_int64)],
    "tts_observe_now": [C.c_void_p, C.c_int, _P(C.c_double)],
    "tts_get_spins": [C.c_void_p, C.c_int, _P(C.c_double)],
    "tts_set_spins": [C.c_void_p, C.c_int, _P(C.c_double)],
    "tts_get_all_spins": [C.c_void_p, _P(C.c_double)],
    "tts_set_all_spins": [C.c_void_p, _P(C.c_double)],
    "tts_instance_size": [C.c_void_p, C.c_int, _P(C.c_int64), _P(C.c_int)],
    "tts_get_species": [C.c_void_p, C.c_int, _P(C.c_int)],
    "tts_get_colours": [C.c_void_p, C.c_int, _P(C.c_int)],
    "tts_get_ttm": [C.c_void_p, C.c_int, _P(C.c_double), _P(C.c_double), _P(C.c_double)],
    "tts_set_ttm_state": [C.c_void_p, C.c_int, _P(C.c_double), _P(C.c_double)],
    "tts_get_step": [C.c_void_p, _P(C.c_int64)],
    "tts_set_step": [C.c_void_p, C.c_int64],
    "tts_get_state": [C.c_void_p, C.c_void_p, _P(C.c_size_t)],
    "tts_set_state": [C.c_void_p, C.c_void_p, C.c_size_t],
    "tts_info": [C.c_void_p, _P(tts_info_t)],
    "tts_profile_enable": [C.c_void_p, C.c_int],
    "tts_profile_read": [C.c_void_p, _P(C.c_double), _P(C.c_int64), _P(C.c_int64)],
    "tts_autotune": [C.c_void_p, C.c_int, _P(C.c_int), _P(C.c_int)],
    "tts_set_config": [C.c_void_p, C.c_int, _P(C.c_int), _P(C.c_int)],
    "tts_read_spins_async": [C.c_void_p, C.c_void_p, C.c_size_t],
    "tts_write_spins_async": [C.c_void_p, C.c_void_p, C.c_size_t],
    "tts_set_lattice": [C.c_void_p, _P(tts_lattice_desc)],
    "tts_get_positions": [C.c_void_p, C.c_int, _P(C.c_double)],
    "tts_get_velocities": [C.c_void_p, C.c_int, _P(C.c_double)],
    "tts_ttm_advance_noalloc": [_P(tts_ttm_desc), _P(C.c_double), C.c_double, C.c_int64, C.c_void_p,
                                C.c_void_p, C.c_void_p, C.c_void_p],
    "tts_health": [C.c_void_p, _P(C.c_uint)],
    "tts_selftest_wait": [C.c_void_p, C.c_int64],
}

HEALTH = {"nonfinite": 1, "timeout": 2, "skin": 4, "colour": 8, "overflow": 16}

_LIB = None


def load():
    """Load libtts.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libtts.so is not built: run python -m paper_2608_18541_b300.build "
                              "(no CPU fallback exists)")
        L = C.CDLL(LIB_PATH)
        for name, args in _SIG.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.tts_last_error.argtypes = []
        L.tts_last_error.restype = C.c_char_p
        _LIB = L
    return _LIB


def _check(code):
    if code != TTS_OK:
        raise TTSError(code, load().tts_last_error().decode())


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def make_desc(sysd, precision=64, engine="auto", obs_capacity=0, instance_base=0):
    """Marshal a workload dictionary into a tts_system_desc (plus arrays that
    must stay alive while the struct is used)."""
    d = tts_system_desc()
    keep = []
    d.lattice = LATTICE[sysd["lattice"]]
    d.nx, d.ny, d.nz = int(sysd.get("nx", 1)), int(sysd.get("ny", 1)), int(sysd.get("nz", 1))
    d.a = float(sysd.get("a", 1.0))
    if sysd["lattice"] == "cluster":
        pos = np.ascontiguousarray(sysd["positions"], dtype=np.float64).reshape(-1)
        spc = np.ascontiguousarray(sysd.get("species", np.zeros(pos.size // 3)), dtype=np.int32)
        keep += [pos, spc]
        d.n_explicit = pos.size // 3
        d.pos_explicit = _dp(pos)
        d.species_explicit = _ip(spc)
    ns = int(sysd["nspecies"])
    d.nspecies = ns
    for t in range(ns):
        d.mu_muB[t] = float(sysd["mu"][t])
        d.K[t] = float(sysd["K"][t])
        d.alpha[t] = float(sysd["alpha"][t])
        for k in range(3):
            d.init_dir[t][k] = float(sysd["init_dir"][t][k])
        for u in range(ns):
            e = sysd["exch"][t][u]
            x = d.exch[t][u]
            x.kind = EXCH[e["kind"]]
            x.J1 = float(e.get("J1", 0.0))
            x.J2 = float(e.get("J2", 0.0))
            x.J3 = float(e.get("J3", 1.0))
            x.rc = float(e.get("rc", 0.0))
    d.frac1 = float(sysd.get("frac1", 0.0))
    for k in range(3):
        d.axis[k] = float(sysd["axis"][k])
        d.B[k] = float(sysd["B"][k])
    d.dt = float(sysd["dt"])
    d.T_bath = float(sysd.get("T_bath", 0.0))
    d.seed = int(sysd["seed"])
    d.precision = int(precision)
    d.sample_every = int(sysd.get("sample_every", 0))
    d.obs_capacity = int(obs_capacity)
    d.engine = ENGINE[engine] if isinstance(engine, str) else int(engine)
    d.instance_base = int(instance_base)
    d.sweep = {"symmetric": 0, "merged": 1}[sysd.get("sweep", "symmetric")]
    d.colour_rc = float(sysd.get("colour_rc", 0.0))
    inst = sysd.get("instances")
    if inst:
        d.n_instances = len(inst)
        cells = np.array([[i.get("nx", d.nx), i.get("ny", d.ny), i.get("nz", d.nz)] for i in inst],
                         dtype=np.int32).reshape(-1)
        frac = np.array([i.get("frac1", d.frac1) for i in inst], dtype=np.float64)
        keep += [cells, frac]
        d.inst_cells = _ip(cells)
        d.inst_frac1 = _dp(frac)
        if any("peak_Te" in i for i in inst):
            pk = np.array([i["peak_Te"] for i in inst], dtype=np.float64)
            keep.append(pk)
            d.inst_peak_Te = _dp(pk)
        if any("fwhm" in i for i in inst):
            fw = np.array([i["fwhm"] for i in inst], dtype=np.float64)
            keep.append(fw)
            d.inst_fwhm = _dp(fw)
        if any("T_bath" in i for i in inst):
            tb = np.array([float(i.get("T_bath", sysd.get("T_bath", 0.0))) for i in inst], dtype=np.float64)
            keep.append(tb)
            d.inst_T_bath = _dp(tb)
    else:
        d.n_instances = 1
    return d, keep


def make_ttm(t):
    x = tts_ttm_desc()
    for k in range(3):
        x.cells[k] = int(t["cells"][k])
    x.gamma_e = float(t["gamma_e"])
    x.C_l = float(t["C_l"])
    x.G = float(t["G"])
    x.kappa_e = float(t.get("kappa_e", 0.0))
    x.T0 = float(t["T0"])
    x.source = SOURCE[t.get("source", "none")]
    x.peak_Te = float(t.get("peak_Te", 0.0))
    x.P0 = float(t.get("P0", 0.0))
    x.fwhm = float(t.get("fwhm", 1e-13))
    x.t0 = float(t.get("t0", -1.0))
    x.spatial = SPATIAL[t.get("spatial", "uniform")]
    x.sigma_xy = float(t.get("sigma_xy", 1.0))
    x.depth_z = float(t.get("depth_z", 1.0))
    return x


class System:
    """A system of one or more instances on the GPU (tts_create_system)."""

    def __init__(self, sysd, ttm=None, precision=64, engine="auto", stream=None, obs_capacity=0,
                 instance_base=0, lattice=None):
        L = load()
        if lattice is not None and engine == "auto":
            engine = "general"
        d, keep = make_desc(sysd, precision, engine, obs_capacity, instance_base)
        h = C.c_void_p()
        _check(L.tts_create_system(C.byref(d), C.c_void_p(stream or 0), C.byref(h)))
        self._h = h
        self.precision = precision
        self.ttm_cells = 0                 # cells of every instance's TTM grid (0: none)
        info = self.info()
        self.n_total = info.n_total
        self.n_instances = info.n_instances
        self.engine = ENGINE_NAME.get(info.engine, info.engine)
        self.sizes = []
        for i in range(self.n_instances):
            n = C.c_int64()
            k = C.c_int()
            _check(L.tts_instance_size(self._h, i, C.byref(n), C.byref(k)))
            self.sizes.append((n.value, k.value))
        if lattice is not None:
            self.set_lattice(lattice)
        if ttm is not None:
            self.set_ttm_grid(ttm)

    def close(self):
        if getattr(self, "_h", None) and _LIB is not None:
            _LIB.tts_destroy(self._h)
            self._h = None

    __del__ = close

    # -- names follow the C ABI --------------------------------------------
    def set_ttm_grid(self, ttm):
        t = make_ttm(ttm)
        _check(load().tts_set_ttm_grid(self._h, C.byref(t)))
        self.ttm_cells = int(t.cells[0]) * int(t.cells[1]) * int(t.cells[2])

    def step(self, n):
        _check(load().tts_step(self._h, int(n)))

    def sync(self):
        _check(load().tts_sync(self._h))

    def observables(self, inst=0, max_samples=None):
        cap = max_samples if max_samples is not None else 1 << 16
        out = np.empty((cap, NOBS))
        n = C.c_int64()
        _check(load().tts_observables(self._h, int(inst), _dp(out), cap, C.byref(n)))
        return out[:n.value].copy()

    def observe_now(self, inst=0):
        out = np.empty(NOBS)
        _check(load().tts_observe_now(self._h, int(inst), _dp(out)))
        return out

    def get_spins(self, inst=0):
        out = np.empty((self.sizes[inst][0], 3))
        _check(load().tts_get_spins(self._h, int(inst), _dp(out)))
        return out

    def set_spins(self, s, inst=0):
        a = np.ascontiguousarray(s, dtype=np.float64).reshape(self.sizes[inst][0], 3)
        _check(load().tts_set_spins(self._h, int(inst), _dp(a)))

    def get_all_spins(self, out=None):
        if out is None:
            out = np.empty((self.n_total, 3))
        _check(load().tts_get_all_spins(self._h, _dp(out)))
        return out

    def set_all_spins(self, s):
        a = np.ascontiguousarray(s, dtype=np.float64).reshape(self.n_total, 3)
        _check(load().tts_set_all_spins(self._h, _dp(a)))

    def read_spins_async(self, out):
        """tts_read_spins_async into a C-contiguous (n_total, 3) array of the
        system's precision (page-locked for full speed); valid after sync()."""
        self._check_io(out)
        _check(load().tts_read_spins_async(self._h, C.c_void_p(out.ctypes.data), C.c_size_t(out.nbytes)))

    def write_spins_async(self, src):
        """tts_write_spins_async from a C-contiguous (n_total, 3) array of the
        system's precision; src must stay untouched until sync()."""
        self._check_io(src)
        _check(load().tts_write_spins_async(self._h, C.c_void_p(src.ctypes.data), C.c_size_t(src.nbytes)))

    def _check_io(self, a):
        dt = np.float32 if self.precision == 32 else np.float64
        if a.dtype != dt or a.shape != (self.n_total, 3) or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("expected a C-contiguous (%d, 3) %s array" % (self.n_total, np.dtype(dt).name))

    def get_species(self, inst=0):
        out = np.empty(self.sizes[inst][0], dtype=np.int32)
        _check(load().tts_get_species(self._h, int(inst), _ip(out)))
        return out

    def get_colours(self, inst=0):
        out = np.empty(self.sizes[inst][0], dtype=np.int32)
        _check(load().tts_get_colours(self._h, int(inst), _ip(out)))
        return out

    def get_ttm(self, inst=0, ncells=None):
        # tts_get_ttm writes every cell of the instance's grid
        nc = max(self.ttm_cells, 1)
        if ncells is not None and ncells != nc:
            raise ValueError("the grid has %d cells, not %d" % (nc, ncells))
        Te = np.empty(nc)
        Tl = np.empty(nc)
        P0 = C.c_double()
        _check(load().tts_get_ttm(self._h, int(inst), _dp(Te), _dp(Tl), C.byref(P0)))
        return Te, Tl, P0.value

    def set_ttm_state(self, Te, Tl, inst=0):
        Te = np.ascontiguousarray(Te, dtype=np.float64)
        Tl = np.ascontiguousarray(Tl, dtype=np.float64)
        _check(load().tts_set_ttm_state(self._h, int(inst), _dp(Te), _dp(Tl)))

    def get_step(self):
        v = C.c_int64()
        _check(load().tts_get_step(self._h, C.byref(v)))
        return v.value

    def set_step(self, n):
        _check(load().tts_set_step(self._h, int(n)))

    def get_state(self):
        L = load()
        n = C.c_size_t()
        _check(L.tts_get_state(self._h, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        _check(L.tts_get_state(self._h, buf, C.byref(n)))
        return buf.raw[:n.value]

    def set_state(self, blob):
        buf = C.create_string_buffer(blob, len(blob))
        _check(load().tts_set_state(self._h, buf, len(blob)))

    def info(self):
        i = tts_info_t()
        _check(load().tts_info(self._h, C.byref(i)))
        return i

    def set_lattice(self, lat):
        x = tts_lattice_desc()
        for name, _ in tts_lattice_desc._fields_:
            if name == "skin":
                x.skin = float(lat.get("skin", 1.0))
            else:
                setattr(x, name, lat[name])
        _check(load().tts_set_lattice(self._h, C.byref(x)))

    def get_positions(self, inst=0):
        out = np.empty((self.sizes[inst][0], 3))
        _check(load().tts_get_positions(self._h, int(inst), _dp(out)))
        return out

    def get_velocities(self, inst=0):
        out = np.empty((self.sizes[inst][0], 3))
        _check(load().tts_get_velocities(self._h, int(inst), _dp(out)))
        return out

    def autotune(self, probe_steps=20):
        """tts_autotune: returns (chosen configuration, configurations offered)."""
        c, n = C.c_int(), C.c_int()
        _check(load().tts_autotune(self._h, int(probe_steps), C.byref(c), C.byref(n)))
        return c.value, n.value

    def set_config(self, index=-1):
        """tts_set_config: select launch configuration `index` (-1: none);
        returns (configuration in use, configurations offered)."""
        c, n = C.c_int(), C.c_int()
        _check(load().tts_set_config(self._h, int(index), C.byref(c), C.byref(n)))
        return c.value, n.value

    def engine_now(self):
        """Engine in use now (it can change when a TTM grid is attached)."""
        return ENGINE_NAME.get(self.info().engine, self.info().engine)

    def profile_enable(self, on=True):
        _check(load().tts_profile_enable(self._h, 1 if on else 0))

    def health(self):
        """tts_health: the raw device health word (TTS_HEALTH_* bits, see HEALTH)."""
        b = C.c_uint()
        _check(load().tts_health(self._h, C.byref(b)))
        return b.value

    def selftest_wait(self, limit_ns):
        """tts_selftest_wait: a bounded device wait that is made to run out."""
        _check(load().tts_selftest_wait(self._h, int(limit_ns)))

    def profile_read(self):
        ms = C.c_double()
        st = C.c_int64()
        ss = C.c_int64()
        _check(load().tts_profile_read(self._h, C.byref(ms), C.byref(st), C.byref(ss)))
        return ms.value, st.value, ss.value


def ttm_advance_noalloc(ttm, box_ang, dt, step, dev_Te, dev_Tl, dev_deposited=0, stream=0):
    """tts_ttm_advance_noalloc: one TTM step on caller-owned device buffers
    (device addresses as ints), allocating nothing.  ttm["P0"] is the source
    power used as given."""
    t = make_ttm(ttm)
    box = (C.c_double * 3)(*[float(v) for v in box_ang])
    _check(load().tts_ttm_advance_noalloc(C.byref(t), box, float(dt), int(step), C.c_void_p(dev_Te),
                                          C.c_void_p(dev_Tl), C.c_void_p(dev_deposited or 0),
                                          C.c_void_p(stream or 0)))


def create_system(sysd, ttm=None, precision=64, engine="auto", stream=None, obs_capacity=0,
                  instance_base=0, lattice=None):
    """tts_create_system (+ tts_set_lattice, tts_set_ttm_grid when given)."""
    return System(sysd, ttm, precision, engine, stream, obs_capacity, instance_base, lattice)
