"""The fused symmetric sweep of the FP32 checker engine (checker_sweep_kernel):
the three colour passes of a step in one launch, a wavefront along z with
the planes in flight in shared memory.  Every site sees the same inputs,
noise and arithmetic as in the three separate passes, so the spins must be
bitwise those of the separate-pass kernel, for every fusion depth (z segments
per instance) offered, cluster shape, instance count, call length and
checkpoint in between; and within the
2e-5 FP32 bar of the FP64 oracle over 200 steps."""
import numpy as np
import pytest

import oracle as O
import paper_2608_18541_b300 as P
from paper_2608_18541_b300 import workloads as W

pytestmark = pytest.mark.gpu

FS = 1e-15


def _launches_per_step(g, n=4):
    g.set_step(1000)                  # the same sampling phase for every measurement
    a = g.info().kernel_launches
    g.profile_enable(True)            # every kernel its own graph node, so that each is counted
    g.step(n)
    g.sync()
    g.profile_enable(False)
    return (g.info().kernel_launches - a) / n


def _fused_and_separate(g):
    """The fused sweep configurations (the last ones offered, one per fusion
    depth: one spin kernel a step) and the default separate-pass
    configuration (three pass launches a step per instance chain)."""
    cur, n = g.set_config(-1)
    assert cur == 0 and n >= 2
    k = []
    for c in range(n):
        g.set_config(c)
        k.append(_launches_per_step(g))
    g.set_config(0)
    fused = []
    for c in range(n - 1, 0, -1):
        if k[c] != min(k):            # one spin kernel a step: the fewest launches
            break
        fused.append(c)
    assert fused and fused[0] == n - 1
    assert k[0] - min(k) >= 2
    return fused, 0


@pytest.mark.parametrize("shape,ninst,ttm", [
    ((16, 16, 16), 1, "cell"),
    ((32, 32, 32), 2, "spot"),
    ((24, 16, 20), 3, "cell"),
    ((64, 64, 64), 1, "spot"),
])
def test_fused_sweep_is_bitwise_the_separate_passes(shape, ninst, ttm):
    nx, ny, nz = shape
    sysd = W.gdfeco_sc(nx, sample_every=7)
    sysd["instances"] = [{"nx": nx, "ny": ny, "nz": nz, "frac1": 0.25} for _ in range(ninst)]
    t = W.ttm_single_cell(1800.0, 20 * FS) if ttm == "cell" else W.ttm_xy_spot(4, 1800.0, 20 * FS, sigma_xy=12.0)
    g = P.System(sysd, t, precision=32, engine="checker")
    assert g.engine == "checker"
    fused, sep = _fused_and_separate(g)
    assert len(fused) >= 2            # fusion depths: z segments per instance
    g.set_step(0)
    start = g.get_state()
    runs = {}
    for c in fused + [sep]:
        g.set_state(start)
        g.set_config(c)
        g.step(13)                    # odd: the state ends in the second buffer
        mid = g.get_state()
        g.step(1)
        g.set_state(mid)              # resume from a checkpoint taken mid-way
        g.step(20)
        runs[c] = ([g.get_spins(i) for i in range(ninst)], g.observables(0), g.get_ttm(0)[0])
    for c in fused:
        for i in range(ninst):
            assert np.array_equal(runs[c][0][i], runs[sep][0][i]), (c, i)
        assert np.array_equal(runs[c][1], runs[sep][1]), c
        assert np.array_equal(runs[c][2], runs[sep][2]), c


def test_fused_sweep_matches_oracle_200_steps():
    sysd = W.gdfeco_sc(16, sample_every=50)
    sysd["instances"] = [{"nx": 16, "ny": 16, "nz": 16, "frac1": f} for f in (0.2, 0.3)]
    ttm = W.ttm_xy_spot(4, 1800.0, 20 * FS, sigma_xy=12.0)
    g = P.System(sysd, ttm, precision=32, engine="checker")
    g.set_config(g.set_config(-1)[1] - 1)          # the fused sweep
    g.step(120)
    g.step(80)
    for i in range(2):
        o = O.Oracle(sysd, ttm, instance=i, index=i)
        o.step(200)
        assert np.abs(g.get_spins(i) - o.spins()).max() <= 2e-5


def test_fused_sweep_full_size_instance_against_separate_passes():
    # the benchmark's instance shape (clusters of 16 CTAs, two z segments)
    sysd, ttm = W.config_gdfeco_large(128, 1)
    g = P.System(dict(sysd, sample_every=0), ttm, precision=32, engine="checker")
    fused, sep = _fused_and_separate(g)
    g.set_step(0)
    start = g.get_state()
    out = []
    for c in [fused[0], sep]:
        g.set_state(start)
        g.set_config(c)
        g.step(5)
        out.append(g.get_spins(0))
    assert np.array_equal(out[0], out[1])
