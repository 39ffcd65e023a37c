"""Oracle pins of the merged sweep (the leapfrog form of the symmetric
splitting, paper Sec. II.A): the trailing half-pass A_0(dt/2) of a step and
the leading half-pass of the next are one full-step pass A_0(dt).

- Under a field that does not depend on the spin itself (no anisotropy) and
  without noise, the frozen-field flow composes exactly, A_0(h/2) A_0(h/2) =
  A_0(h), so the merged and symmetric sweeps give the same trajectory up to
  rounding.  A bridge pass with the wrong length, a missing or doubled close
  or a wrong pass order breaks that.
- With anisotropy the bridge differs from two halves at O(dt^3) per step: the
  merged sweep is still second order against an accurate ODE solution.
- A call of one step closes at once, so single-step calls are exactly the
  symmetric sweep; the sweep closes at sampling steps, so sampled states are
  at whole steps.
- Thermal equilibrium under the bridge's full-step noise amplitude: the
  two-spin law <s1.s2> = coth(beta J) - 1/(beta J)."""
import numpy as np
from scipy.integrate import solve_ivp

import oracle as O
from paper_2608_18541_b300 import workloads as W

from test_oracle_dynamics import FS, _cluster_case, _llg_rhs_factory
from test_oracle_statistics import KB, MUB, GAMMA, _time_average, langevin


def _no_onsite(sysd):
    s = dict(sysd, K=[0.0] * sysd["nspecies"], T_bath=0.0, B=[0.3, -0.2, 2.0], dt=1.0 * FS)
    s["alpha"] = [0.05] * sysd["nspecies"]
    s["init_dir"] = [[0.3, 0.1, 0.95], [-0.2, 0.4, -0.9]]
    return s


def test_merged_equals_symmetric_without_onsite_terms():
    for base in (W.gdfeco_sc(6), W.bcc_fe(3)):
        sysd = _no_onsite(base)
        a = O.Oracle(dict(sysd, sweep="symmetric"))
        b = O.Oracle(dict(sysd, sweep="merged"))
        assert a.ncolours >= 2
        a.step(40)
        b.step(40)
        d = np.abs(a.spins() - b.spins()).max()
        assert d < 1e-12, (a.ncolours, d)
        # and the dynamics did something
        assert np.abs(a.spins() - O.Oracle(sysd).spins()).max() > 1e-3


def test_single_step_calls_are_the_symmetric_sweep():
    sysd = W.gdfeco_sc(6, T=300.0)
    ttm = W.ttm_single_cell(1500.0, 20 * FS)
    a = O.Oracle(dict(sysd, sweep="symmetric"), ttm)
    b = O.Oracle(dict(sysd, sweep="merged"), ttm)
    a.step(12)
    for _ in range(12):
        b.step(1)
    assert np.array_equal(a.spins(), b.spins())


def test_merged_sweep_closes_at_sampling_steps():
    sysd = W.gdfeco_sc(6, T=300.0, sample_every=5)
    ttm = W.ttm_single_cell(1500.0, 20 * FS)
    a = O.Oracle(dict(sysd, sweep="merged"), ttm)
    b = O.Oracle(dict(sysd, sweep="merged"), ttm)
    a.step(20)                       # closes at steps 5, 10, 15, 20
    for _ in range(4):
        b.step(5)                    # closes at the same steps
    assert np.array_equal(a.samples(), b.samples())
    assert np.array_equal(a.spins(), b.spins())
    c = O.Oracle(dict(sysd, sweep="symmetric"), ttm)
    c.step(20)
    assert not np.array_equal(a.spins(), c.spins())     # the bridges did change the path


def _run_cluster_merged(dt, tend, alpha, K, B):
    pos, J, init = _cluster_case()
    sysd = W.cluster(pos, J=J, rc=3.0, mu=2.0, B=B, T=0.0, alpha=alpha, dt=dt, K=K)
    sysd["sweep"] = "merged"
    o = O.Oracle(sysd)
    o.set_spins(init)
    o.step(int(round(tend / dt)))
    return o.spins()


def test_merged_sweep_is_second_order_against_ode_reference():
    pos, J, init = _cluster_case()
    alpha, K, B = 0.1, 2e-22, (0.0, 3.0, 20.0)
    tend = 60 * FS
    rhs = _llg_rhs_factory(pos, J, 3.0, 2.0, K, [0, 0, 1], B, alpha)
    ref = solve_ivp(rhs, (0, tend), init.reshape(-1), method="DOP853", rtol=1e-13, atol=1e-15).y[:, -1]
    ref = ref.reshape(3, 3)
    errs = [np.abs(_run_cluster_merged(dt, tend, alpha, K, B) - ref).max() for dt in (2.0 * FS, 1.0 * FS, 0.5 * FS)]
    o1 = np.log2(errs[0] / errs[1])
    o2 = np.log2(errs[1] / errs[2])
    assert 1.85 < o1 < 2.15 and 1.85 < o2 < 2.15, (errs, o1, o2)


def test_merged_two_spin_thermal_law():
    T, betaJ, mu, alpha = 10.0, 2.0, 2.0, 1.0
    J = betaJ * KB * T
    npair = 512
    pos = np.zeros((2 * npair, 3))
    pos[0::2, 0] = np.arange(npair) * 20.0
    pos[1::2, 0] = np.arange(npair) * 20.0 + 2.5
    sysd = W.cluster(pos, J=J, rc=3.0, mu=mu, T=T, alpha=alpha, dt=1.0 * FS, seed=9)
    sysd["sweep"] = "merged"
    o = O.Oracle(sysd)
    Bex = J / (mu * MUB)
    nt = int(round((1 + alpha ** 2) / (alpha * GAMMA * Bex) / (1.0 * FS)))

    def dots(o):
        s = o.spins()
        return (s[0::2] * s[1::2]).sum(1)

    per_pair = _time_average(o, 6 * nt, 20, nt // 2, dots)
    m = per_pair.mean()
    se = per_pair.std(ddof=1) / np.sqrt(npair)
    assert abs(m - langevin(betaJ)) < 3 * se, (m, langevin(betaJ), se)
