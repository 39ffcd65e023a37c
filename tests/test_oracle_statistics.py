"""Oracle pins: thermal equilibrium laws that fix the noise variance, its
1/sqrt(mu) scaling (Sec. II.C), the placement of (1 + alpha^2) and the
Stratonovich reading.  Each run averages many independent spins or pairs;
standard errors come from per-spin (per-pair) time averages, which are
independent of each other."""
import numpy as np
import pytest

import oracle as O
from paper_2608_18541_b300 import workloads as W

KB = 1.380649e-23
MUB = 9.2740100783e-24
GAMMA = 1.76085963023e11
FS = 1e-15


def langevin(x):
    return 1.0 / np.tanh(x) - 1.0 / x


def _time_average(o, n_eq, n_samp, every, fn):
    o.step(n_eq)
    acc = None
    for _ in range(n_samp):
        o.step(every)
        v = fn(o)
        acc = v if acc is None else acc + v
    return acc / n_samp


@pytest.mark.parametrize("mu,alpha", [(1.92, 1.0), (7.63, 1.0), (1.92, 0.1), (7.63, 0.1)])
def test_single_spin_langevin_law(mu, alpha):
    # <s_z> = coth(x) - 1/x, x = mu B / (k_B T), for independent spins in a
    # field at bath temperature T; B = 10 T, T = 10 K gives x = 1.29 (Fe) and
    # 5.12 (Gd).  An extra 2 pi in the variance, a 1/mu instead of 1/sqrt(mu)
    # amplitude or a misplaced (1 + alpha^2) each moves <s_z> by many SE.
    B, T = 10.0, 10.0
    dt = 1.0 * FS if alpha >= 1.0 else 3.0 * FS
    tau = (1 + alpha ** 2) / (alpha * GAMMA * B)          # longitudinal relaxation time scale
    nt = int(round(tau / dt))
    sysd = W.single_spins(1024, mu=mu, B=(0, 0, B), T=T, alpha=alpha, dt=dt, seed=77)
    o = O.Oracle(sysd)
    per_spin = _time_average(o, 6 * nt, 20, nt // 2, lambda o: o.spins()[:, 2])
    m = per_spin.mean()
    se = per_spin.std(ddof=1) / np.sqrt(per_spin.size)
    x = mu * MUB * B / (KB * T)
    assert abs(m - langevin(x)) < 4 * se, (m, langevin(x), se)


def test_two_spin_thermal_law():
    # isolated pairs with E = -J s1.s2: <s1.s2> = coth(beta J) - 1/(beta J)
    T, betaJ, mu, alpha = 10.0, 2.0, 2.0, 1.0
    J = betaJ * KB * T
    npair = 512
    pos = np.zeros((2 * npair, 3))
    pos[0::2, 0] = np.arange(npair) * 20.0
    pos[1::2, 0] = np.arange(npair) * 20.0 + 2.5
    sysd = W.cluster(pos, J=J, rc=3.0, mu=mu, T=T, alpha=alpha, dt=1.0 * FS, seed=5)
    o = O.Oracle(sysd)
    assert o.ncolours == 2
    Bex = J / (mu * MUB)
    nt = int(round((1 + alpha ** 2) / (alpha * GAMMA * Bex) / (1.0 * FS)))

    def dots(o):
        s = o.spins()
        return (s[0::2] * s[1::2]).sum(1)

    per_pair = _time_average(o, 6 * nt, 20, nt // 2, dots)
    m = per_pair.mean()
    se = per_pair.std(ddof=1) / np.sqrt(npair)
    assert abs(m - langevin(betaJ)) < 4 * se, (m, langevin(betaJ), se)


def _sublattice_temperatures(noise_mu_power):
    sysd = W.gdfeco_sc(8, alpha=0.1, dt=0.2 * FS, T=300.0, seed=21)
    o = O.Oracle(sysd, noise_mu_power=noise_mu_power)
    o.step(9000)
    blocks = []
    for _ in range(12):
        acc = np.zeros(2)
        for _ in range(15):
            o.step(100)
            acc += o.observe()[13:15]
        blocks.append(acc / 15)
    blocks = np.array(blocks)
    return blocks.mean(0), blocks.std(0, ddof=1) / np.sqrt(len(blocks))


def test_mu_fdt_equilibrates_both_sublattices():
    # Sec. II.C: with noise ~ 1/sqrt(mu) both sublattices of a two-species
    # magnet at one bath temperature equilibrate to it (spin temperature
    # sum |s x H|^2 / (2 k_B sum s.H) per sublattice)
    Ts, se = _sublattice_temperatures(0.5)
    for k in range(2):
        assert abs(Ts[k] - 300.0) < max(4 * se[k], 0.03 * 300.0), (Ts, se)


def test_without_mu_fdt_heavy_sublattice_runs_cold():
    # the paper's failure mode, planted in the oracle: noise rescaled by
    # mu_ref/mu with the torque (no mu_fdt) leaves the Gd sublattice cold
    Ts, se = _sublattice_temperatures(1.0)
    assert Ts[1] < 0.8 * 300.0, (Ts, se)
    assert abs(Ts[0] - 300.0) < 0.2 * 300.0
