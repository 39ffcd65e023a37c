"""Bulk asynchronous spin I/O (tts_read_spins_async / tts_write_spins_async):
canonical atom order and the system's precision, the same values as the
synchronous per-instance calls, and a written state that steps exactly like
one set through tts_set_all_spins."""
import numpy as np
import pytest

import paper_2608_18541_b300 as P
from paper_2608_18541_b300 import workloads as W

pytestmark = pytest.mark.gpu
FS = 1e-15


def _systems():
    s = W.gdfeco_sc(8)
    s["instances"] = [{"nx": 8, "ny": 8, "nz": 8, "frac1": 0.25}, {"nx": 8, "ny": 8, "nz": 8, "frac1": 0.3}]
    return [
        ("checker", 32, s, W.ttm_single_cell(1500.0, 20 * FS)),
        ("general", 64, W.bcc_fe(4), None),
        ("resident", 32, W.config_ensemble(n_peak=1, n_dur=1, n_real=3, lmin=5, lmax=7)[0],
         W.config_ensemble(n_peak=1, n_dur=1, n_real=3, lmin=5, lmax=7)[1]),
    ]


@pytest.mark.parametrize("engine,prec,sysd,ttm", _systems())
def test_bulk_io_matches_sync_calls_and_steps_identically(engine, prec, sysd, ttm):
    dt = np.float32 if prec == 32 else np.float64
    g = P.System(sysd, ttm, precision=prec, engine=engine)
    g.step(7)
    buf = np.empty((g.n_total, 3), dtype=dt)
    g.read_spins_async(buf)
    g.sync()
    assert np.array_equal(buf.astype(np.float64), g.get_all_spins())
    # a new state set through the synchronous call on one system, carried
    # over with the bulk calls to another: both then step identically
    rng = np.random.default_rng(5)
    v = rng.normal(size=(g.n_total, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    h = P.System(sysd, ttm, precision=prec, engine=engine)
    h.step(7)
    h.set_all_spins(v)
    state = np.empty((g.n_total, 3), dtype=dt)
    h.read_spins_async(state)
    h.sync()
    g.write_spins_async(state)
    g.sync()
    assert np.array_equal(g.get_all_spins(), state.astype(np.float64))
    g.step(9)
    h.step(9)
    assert np.array_equal(g.get_all_spins(), h.get_all_spins())
    with pytest.raises(ValueError):
        g.read_spins_async(np.empty((g.n_total, 2), dtype=dt))
