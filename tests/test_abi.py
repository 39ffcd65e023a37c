"""The C-ABI library loads and exports every entry point include/tts.h
declares; descriptor errors come back as TTS_ERR_ARG before any CUDA call
(no GPU needed)."""
import os
import re

import pytest

import paper_2608_18541_b300 as P
from paper_2608_18541_b300 import build as B
from paper_2608_18541_b300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        names += re.findall(r"TTS_API\s+[\w\s\*]*?\b(tts_\w+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return P.load()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("tts_create_system", "tts_destroy", "tts_set_ttm_grid", "tts_step", "tts_sync",
                     "tts_observables", "tts_get_spins", "tts_set_spins", "tts_get_state",
                     "tts_set_state", "tts_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_signatures_cover_the_header(lib):
    declared = set(_declared()) - {"tts_last_error"}
    assert declared == set(P._SIG)


@pytest.mark.parametrize("mutate,msg", [
    (lambda d: d.update(nspecies=3, mu=[1, 1, 1], K=[0] * 3, alpha=[0] * 3, init_dir=[[0, 0, 1]] * 3,
                        exch=[[W.ZERO_EXCH] * 3] * 3), "nspecies"),
    (lambda d: d.update(dt=0.0), "dt"),
    (lambda d: d.update(nx=2), "twice the cutoff"),
    (lambda d: d.update(mu=[0.0]), "moments"),
    (lambda d: d.update(frac1=1.5), "fraction"),
])
def test_bad_descriptors_are_rejected_on_the_host(lib, mutate, msg):
    d = W.bcc_fe(4)
    mutate(d)
    with pytest.raises((P.TTSError, IndexError)) as ei:
        P.System(d)
    if isinstance(ei.value, P.TTSError):
        assert ei.value.code == -1
        assert msg in str(ei.value)


def test_asymmetric_exchange_is_rejected(lib):
    d = W.gdfeco_sc(6)
    d["exch"][0][1] = dict(d["exch"][0][1], J1=-2e-21)
    with pytest.raises(P.TTSError) as ei:
        P.System(d)
    assert ei.value.code == -1 and "symmetric" in str(ei.value)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(P, "LIB_PATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(P, "_LIB", None)
    with pytest.raises(ImportError):
        P.load()


@pytest.mark.parametrize("change,msg", [
    (dict(spatial="xy_gauss", sigma_xy=0.0), "sigma_xy > 0"),
    (dict(spatial="z_exp", depth_z=0.0), "depth_z > 0"),
    (dict(cells=[2 ** 21, 2 ** 21, 2 ** 22]), "at most 65536"),
    (dict(cells=[65537, 1, 1]), "at most 65536"),
    (dict(cells=[41, 40, 40]), "at most 65536"),
    (dict(cells=[0, 4, 4]), ">= 1"),
])
def test_noalloc_arguments_are_checked_on_the_host(lib, change, msg):
    # rejected before any device work: the buffers are never touched
    t = dict(W.ttm_xy_spot(8), source="power", P0=1e20)
    t.update(change)
    with pytest.raises(P.TTSError) as ei:
        P.ttm_advance_noalloc(t, [100.0, 100.0, 100.0], 1e-16, 0, 0x1000, 0x2000)
    assert ei.value.code == -1 and msg in str(ei.value)
