"""Profiled steps (tts_profile_*): the colour passes timed with CUDA events
inside a replayed graph.  Profiling must not change the trajectory, must count
every step and kernel, and the pass time it reports must fit inside the
graph-timed step."""
import numpy as np
import pytest

import paper_2608_18541_b300 as P
from paper_2608_18541_b300 import workloads as W

pytestmark = pytest.mark.gpu

FS = 1e-15


def _system():
    sysd = W.gdfeco_sc(32, sample_every=10)
    sysd["instances"] = [{"nx": 32, "ny": 32, "nz": 32, "frac1": f} for f in (0.2, 0.3)]
    return P.System(sysd, W.ttm_xy_spot(4, 1800.0, 20 * FS, sigma_xy=12.0), precision=32, engine="checker")


def test_profiled_steps_match_graph_steps_bitwise():
    a, b = _system(), _system()
    a.step(25)
    b.profile_enable(True)
    b.step(12)
    b.step(13)
    b.sync()
    ms, steps, spin_steps = b.profile_read()
    b.profile_enable(False)
    assert steps == 25 and spin_steps == 25 * b.n_total
    assert ms > 0.0
    for i in range(2):
        assert np.array_equal(a.get_spins(i), b.get_spins(i))
    assert np.array_equal(a.observables(0), b.observables(0))


def test_profiled_pass_time_fits_the_step():
    import torch
    g = _system()
    st = torch.cuda.current_stream()
    g.step(20)
    g.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    g.step(200)
    e1.record(st)
    torch.cuda.synchronize()
    step_ms = e0.elapsed_time(e1) / 200
    k0 = g.info().kernel_launches
    g.profile_enable(True)
    g.step(200)
    g.sync()
    ms, steps, _ = g.profile_read()
    g.profile_enable(False)
    assert steps == 200
    assert g.info().kernel_launches - k0 >= 200 * 6     # three passes on each of two instance chains
    pass_ms = ms / steps
    assert 0.0 < pass_ms <= 1.25 * step_ms, (pass_ms, step_ms)


def test_mode_switches_at_odd_steps_keep_the_trajectory():
    """The step graphs run the TTM beside the colour passes on noise tables
    alternated by step parity; profiled steps and single-chain configurations
    keep one table.  Switching between them after an odd number of steps must
    leave the trajectory bitwise unchanged."""
    a, b = _system(), _system()
    a.step(31)
    b.step(7)                        # graphs from an even step
    b.profile_enable(True)
    b.step(5)                        # profiled, from an odd step
    b.profile_enable(False)
    b.step(3)                        # graphs from an even step again
    _, n = b.set_config(-1)
    for c in (1, 0, n - 1, 0):       # a single chain, two chains, the last configuration
        b.set_config(c)
        b.step(3)                    # ends on steps 18, 21, 24, 27
    b.step(4)
    assert b.get_step() == 31
    for i in range(2):
        assert np.array_equal(a.get_spins(i), b.get_spins(i))
    assert np.array_equal(a.observables(0), b.observables(0))
