"""Failure detection on the GPU, without a GPU fault: every condition that
the device health word reports is made to happen and must come back through
tts_sync as a status (and through tts_health as its bit), with the context
still usable afterwards.

- a bounded device wait that runs out (a barrier waiting for a transfer that
  is never issued, its limit cut to 50 ms): TTS_ERR_DEVICE_TIMEOUT;
- (a non-finite spin, a NaN written into a checkpoint, is the parity
  tests' case);
- moving lattice, an atom beyond half its skin (a skin of 0.02 A, below the
  initial strain displacement of 0.014 A): TTS_ERR_HEALTH;
- moving lattice, two exchange-coupled atoms of one colour, and more exchange
  neighbours than the table holds: a 35 % local compression of bcc Fe along z
  brings same-colour pairs (4.05 A apart) inside the 3.5 A cutoff and raises
  the neighbour count from 14 to 18 (the oracle counts 288 such pairs and 18
  neighbours for this state); with a colour margin of 5.5 A no pair can join
  one colour, and only the table overflows."""
import numpy as np
import pytest

import paper_2608_18541_b300 as P
from paper_2608_18541_b300 import workloads as W

pytestmark = pytest.mark.gpu

H = P.HEALTH


def _still_usable():
    g = P.System(W.gdfeco_sc(8), precision=32)
    g.step(3)
    g.sync()
    assert g.health() == 0


def test_bounded_wait_times_out():
    g = P.System(W.gdfeco_sc(8), precision=32)
    g.step(2)
    g.sync()
    g.selftest_wait(50_000_000)                  # 50 ms
    with pytest.raises(P.TTSError) as ei:
        g.sync()
    assert ei.value.code == -4                   # TTS_ERR_DEVICE_TIMEOUT
    assert g.health() & H["timeout"]
    with pytest.raises(P.TTSError):
        g.selftest_wait(0)                       # limit out of range
    _still_usable()


def _lattice_system(strain, skin, colour_rc=0.0):
    s = W.bcc_fe(6, T=300.0, alpha=0.1)
    s["colour_rc"] = colour_rc
    lat = W.morse_fe_lattice(T_init=300.0, strain_amp=strain)
    lat["skin"] = skin
    return P.System(s, None, precision=64, lattice=lat)


def test_skin_bit():
    g = _lattice_system(0.005, 0.02)
    g.step(1)
    with pytest.raises(P.TTSError) as ei:
        g.sync()
    assert ei.value.code == -5 and "skin" in str(ei.value)
    assert g.health() & H["skin"]
    _still_usable()


def test_colour_bit():
    g = _lattice_system(0.35, 2.5)
    g.step(1)
    with pytest.raises(P.TTSError) as ei:
        g.sync()
    assert ei.value.code == -5
    bits = g.health()
    assert bits & H["colour"] and not bits & H["skin"]
    _still_usable()


def test_overflow_bit_alone():
    g = _lattice_system(0.35, 2.5, colour_rc=5.5)
    assert g.info().max_colours == 16
    g.step(1)
    with pytest.raises(P.TTSError) as ei:
        g.sync()
    assert ei.value.code == -5 and "neighbours" in str(ei.value)
    bits = g.health()
    assert bits & H["overflow"] and not bits & (H["colour"] | H["skin"])
    _still_usable()


def test_healthy_lattice_stays_clean():
    g = _lattice_system(0.005, 1.4)
    g.step(3)
    g.sync()
    assert g.health() == 0
