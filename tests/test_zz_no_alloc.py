"""The allocation-free TTM advance (tts_ttm_advance_noalloc).

Some callers cannot allocate device memory: code whose device memory is all
owned by another allocator (such as a framework's caching pool) and
latency-critical code that must not call cudaMalloc / cudaFree, which can
synchronise the device.  This entry point advances a TTM grid held in the
caller's own buffers with its scratch in a fixed device array.  Here its
output is checked, over two calls in a row, against the same grid advanced by
tts_step of a system built with tts_create_system / tts_set_ttm_grid.  The
file is named so that pytest collects it last.
"""
import numpy as np
import pytest

import paper_2608_18541_b300 as P
from paper_2608_18541_b300 import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_ttm_advance_matches_system_step_twice():
    import torch

    n = 16
    sysd = W.gdfeco_sc(n, T=300.0)
    ttm = W.ttm_xy_spot(8, 1800.0, 20e-15, sigma_xy=12.0)
    nc = 8 ** 3
    stream = torch.cuda.current_stream()
    g = P.System(sysd, ttm, precision=64, engine="general", stream=stream.cuda_stream)
    start = 255                                   # near the pulse maximum (t0 = 3 sigma_t)
    g.set_step(start)
    Te0, Tl0, P0 = g.get_ttm(0, nc)
    dev_Te = torch.tensor(Te0, dtype=torch.float64, device="cuda")
    dev_Tl = torch.tensor(Tl0, dtype=torch.float64, device="cuda")
    dep = torch.zeros(1, dtype=torch.float64, device="cuda")
    t = dict(ttm, source="power", P0=P0)
    box = [n * 3.52] * 3
    vol = (n * 3.52e-10) ** 3 / nc
    prev_e = (0.5 * 225.0 * Te0 ** 2 + 3.1e6 * Tl0).sum() * vol
    for k in range(2):
        P.ttm_advance_noalloc(t, box, sysd["dt"], start + k, dev_Te.data_ptr(), dev_Tl.data_ptr(),
                              dep.data_ptr(), stream.cuda_stream)
        g.step(1)
        Te, Tl, _ = g.get_ttm(0, nc)
        torch.cuda.synchronize()
        got_Te = dev_Te.cpu().numpy()
        got_Tl = dev_Tl.cpu().numpy()
        assert np.allclose(got_Te, Te, rtol=1e-10, atol=0)
        assert np.allclose(got_Tl, Tl, rtol=1e-10, atol=0)
        assert got_Te.max() > Te0.max()           # the pulse really heated the grid
        # the energy added equals the reported deposit
        e = (0.5 * 225.0 * got_Te ** 2 + 3.1e6 * got_Tl).sum() * vol
        d = float(dep.cpu().item())
        assert d > 0 and abs((e - prev_e) - d) < 1e-9 * d
        prev_e = e


def test_noalloc_rejects_grids_above_the_limit():
    import torch

    t = dict(W.ttm_xy_spot(8), cells=[41, 40, 40], source="power", P0=1e20)
    buf = torch.zeros(41 * 40 * 40, dtype=torch.float64, device="cuda")
    with pytest.raises(P.TTSError) as ei:
        P.ttm_advance_noalloc(t, [100.0, 100.0, 100.0], 1e-16, 0, buf.data_ptr(), buf.data_ptr())
    assert ei.value.code == -1 and "at most 65536" in str(ei.value)
