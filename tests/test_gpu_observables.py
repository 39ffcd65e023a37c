"""Every observable field of the FP32 engines against the FP64 oracle.

The FP32 checker and resident engines compute each site's observable terms
from FP32 spins.  The resident engine sums them in FP64; the checker engine
sums a block's 1024 terms with compensated (TwoSum) FP32 additions, within
2^-40 of the sum of their magnitudes, and the block partials in FP64 (the
per-sublattice magnetisation and energy reductions).  Each field is compared with the oracle's within a bound
propagated from a bound eps on every spin component's error: the rounding of
a given state to FP32 (first test), or the 2e-5 FP32 parity bar after up to
200 steps (second test).  The bounds are worst-case sums over sites, computed
from the oracle's state, its neighbour lists and fields:
  mean s per species, moment-weighted M ........ eps
  exchange energy -sum_{i<j} J s_i.s_j ......... (eps_v + 1e-6) sum_i sum_j |J_ij|
  anisotropy -sum K (s.n)^2 .................... sum_i K (2 eps + eps^2) + 1e-6 sum K
  Zeeman -sum mu B.s ............................ (eps_v + 1e-6) sum_i mu_i |B|
  spin temperature sum|s x H|^2 / (2 k_B sum s.H)  relative: dnum/num + dden/den
with eps_v = sqrt(3) eps the bound on a spin vector's error, 1e-6 a generous
bound on the FP32 rounding of a site's terms relative to their size, and, per
site, the field error b_i = (eps_v sum_j |J_ij| + 2 K eps_v) / mu_i + 1e-6 |B_i|,
e_i = eps_v |B_i| + b_i, dnum = sum mu_i^2 (2 |s x B_i| e_i + e_i^2),
dden = sum mu_i e_i.  Mean T_e and T_l are FP64 on both sides (1e-10)."""
import numpy as np
import pytest

import oracle as O
import paper_2608_18541_b300 as P
from paper_2608_18541_b300 import workloads as W

pytestmark = pytest.mark.gpu

FS = 1e-15
MUB = 9.2740100783e-24


def _tolerances(o, sysd, eps):
    """Per-field bounds (fields 1..16) for spins within eps of the oracle's."""
    s = o.spins()
    sp = o.species()
    n = s.shape[0]
    mu = np.array(sysd["mu"], dtype=float)[sp] * MUB
    K = np.array(sysd["K"], dtype=float)[sp]
    Bext = np.linalg.norm(sysd["B"])
    ev = np.sqrt(3.0) * eps
    sumJ = np.empty(n)
    B = np.empty((n, 3))
    for i in range(n):
        sumJ[i] = np.abs(o.neighbours(i)[1]).sum()
        B[i] = o.field(i)
    Bn = np.linalg.norm(B, axis=1)
    b = (ev * sumJ + 2 * K * ev) / mu + 1e-6 * Bn
    e = ev * Bn + b
    cross = np.linalg.norm(np.cross(s, B), axis=1)
    tol = np.zeros(17)
    tol[1:10] = eps + 1e-9
    tol[10] = (ev + 1e-6) * sumJ.sum()
    tol[11] = (K * (2 * eps + eps * eps)).sum() + 1e-6 * K.sum()
    tol[12] = (ev + 1e-6) * (mu * Bext).sum() + 1e-30
    obs = o.observe()
    for t in (0, 1):
        m = sp == t
        num = (mu[m] ** 2 * cross[m] ** 2).sum()
        den = (mu[m] * np.einsum("ij,ij->i", s[m], B[m])).sum()
        dnum = (mu[m] ** 2 * (2 * cross[m] * e[m] + e[m] ** 2)).sum()
        dden = (mu[m] * e[m]).sum()
        tol[13 + t] = 1.1 * abs(obs[13 + t]) * (dnum / num + dden / abs(den)) + 1e-9
    tol[15:17] = 1e-10 * np.abs(obs[15:17])
    return tol, obs


def _check(got, want, tol, what):
    for k in range(1, 17):
        assert abs(got[k] - want[k]) <= tol[k], (what, k, got[k], want[k], tol[k])


def _random_state(n, species, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    base = np.where(species[:, None] == 0, [0.0, 0.0, 1.0], [0.0, 0.0, -1.0])
    v = base + 0.7 * rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1)[:, None]


@pytest.mark.parametrize("engine", ["checker", "resident"])
def test_fp32_observables_of_a_given_state(engine):
    # the same random state on both sides: the GPU's spins differ from the
    # oracle's by the FP32 rounding of the input (eps = 3e-7 per component)
    sysd = W.gdfeco_sc(12, B=1.0, sample_every=0)
    ttm = W.ttm_single_cell(1200.0, 20 * FS)
    g = P.System(sysd, ttm, precision=32, engine=engine)
    assert g.engine == engine
    o = O.Oracle(sysd, ttm)
    s0 = _random_state(o.n, o.species(), 11)
    g.set_spins(s0)
    o.set_spins(s0)
    tol, want = _tolerances(o, sysd, 3e-7)
    _check(g.observe_now(0), want, tol, "given state")


@pytest.mark.parametrize("engine", ["checker", "resident"])
def test_fp32_observables_along_200_steps(engine):
    # samples every 50 steps (in-step reductions of the engine) against the
    # oracle's, with bounds from the 2e-5 FP32 spin bar at each sample
    sysd = W.gdfeco_sc(12, B=1.0, sample_every=50)
    ttm = W.ttm_single_cell(1200.0, 20 * FS)
    g = P.System(sysd, ttm, precision=32, engine=engine)
    assert g.engine == engine
    o = O.Oracle(sysd, ttm)
    tols = []
    for _ in range(4):
        o.step(50)
        tols.append(_tolerances(o, sysd, 2e-5)[0])
    g.step(200)
    assert np.abs(g.get_spins() - o.spins()).max() <= 2e-5
    gs, osm = g.observables(0), o.samples()
    assert gs.shape == osm.shape == (4, P.NOBS)
    assert np.array_equal(gs[:, 19], osm[:, 19])
    for r in range(4):
        assert gs[r, 0] == osm[r, 0]
        _check(gs[r], osm[r], tols[r], "sample %d" % r)
