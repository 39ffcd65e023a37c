"""Oracle pins: thermal equilibrium laws that fix the noise variance, its
1/sqrt(mu) scaling (Sec. II.C), the placement of (1 + alpha^2) and the
Stratonovich reading.  Each run averages many independent spins or pairs;
standard errors come from per-spin (per-pair) time averages, which are
independent of each other.  Pass rule: within 3 standard errors (a correct
sampler fails one such check with probability 0.27 %; the seeds are fixed, so
the outcome is reproducible)."""
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
    assert abs(m - langevin(x)) < 3 * se, (m, langevin(x), se)


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
    assert abs(m - langevin(betaJ)) < 3 * se, (m, langevin(betaJ), se)


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
        assert abs(Ts[k] - 300.0) < 3 * se[k], (Ts, se)


def test_without_mu_fdt_heavy_sublattice_runs_cold():
    # the paper's failure mode, planted in the oracle: noise rescaled by
    # mu_ref/mu with the torque (no mu_fdt) leaves the Gd sublattice cold
    Ts, se = _sublattice_temperatures(1.0)
    assert Ts[1] < 0.8 * 300.0, (Ts, se)
    assert abs(Ts[0] - 300.0) < 0.2 * 300.0


def _triangle_quadrature(bJ, bK, bB, nc=24, nphi=32):
    """<E>/kT, <s1.s2> and <s1_z> for three unit spins with
    E/kT = -(bJ[0] s1.s2 + bJ[1] s1.s3 + bJ[2] s2.s3) - bK sum (s_i.z)^2 - bB sum s_i.z,
    by quadrature over (S^2)^3: Gauss-Legendre in cos(theta_i), the periodic
    trapezoid rule in phi_2 - phi_1 and phi_3 - phi_1 (the energy does not
    depend on phi_1)."""
    x, w = np.polynomial.legendre.leggauss(nc)
    phi = 2.0 * np.pi * np.arange(nphi) / nphi
    c2, c3 = x[:, None, None, None], x[None, :, None, None]
    w23 = (w[:, None] * w[None, :])[:, :, None, None]
    p2, p3 = phi[None, None, :, None], phi[None, None, None, :]
    s2, s3 = np.sqrt(1 - c2 ** 2), np.sqrt(1 - c3 ** 2)
    d23 = c2 * c3 + s2 * s3 * np.cos(p2 - p3)
    z = e_acc = d12_acc = m_acc = 0.0
    shift = -(abs(bJ[0]) + abs(bJ[1]) + abs(bJ[2]) + 3 * abs(bK) + 3 * abs(bB))   # lowest possible E/kT
    for c1, w1 in zip(x, w):
        s1 = np.sqrt(1 - c1 ** 2)
        d12 = c1 * c2 + s1 * s2 * np.cos(p2)
        d13 = c1 * c3 + s1 * s3 * np.cos(p3)
        e = (-(bJ[0] * d12 + bJ[1] * d13 + bJ[2] * d23) - bK * (c1 ** 2 + c2 ** 2 + c3 ** 2)
             - bB * (c1 + c2 + c3))
        wt = w1 * w23 * np.exp(-(e - shift))
        z += wt.sum()
        e_acc += (e * wt).sum()
        d12_acc += (np.broadcast_to(d12, wt.shape) * wt).sum()
        m_acc += c1 * wt.sum()
    return e_acc / z, d12_acc / z, m_acc / z


def test_triangle_quadrature_reduces_to_two_spin_law():
    # with only the 1-2 bond and no on-site terms, <s1.s2> = coth(bJ) - 1/bJ
    for bJ in (0.5, 2.0):
        _, d12, m = _triangle_quadrature((bJ, 0.0, 0.0), 0.0, 0.0)
        assert abs(d12 - langevin(bJ)) < 1e-10, (d12, langevin(bJ))
        assert abs(m) < 1e-12
    # converged in the grid
    a = _triangle_quadrature((1.5, 1.5, 1.5), 1.0, 0.5)
    b = _triangle_quadrature((1.5, 1.5, 1.5), 1.0, 0.5, nc=32, nphi=48)
    assert np.allclose(a, b, rtol=0, atol=1e-9), (a, b)


def test_three_spin_thermal_equilibrium():
    # isolated equilateral triangles (three colours, so the five-pass
    # symmetric sweep) with exchange, uniaxial anisotropy and a field along z,
    # at bath temperature T: the time averages of E/kT, s1.s2 and s_z over
    # independent triangles match the Boltzmann averages by quadrature.  The
    # slowest mode (the triangle's total spin against the on-site terms) sets
    # the times; the start is isotropic.  At dt = 1 fs the energy read about
    # one SE low (the integrator's O(dt^2) bias of the stationary law), at
    # 0.5 fs a fifth of that; a bath 5 % too warm reads 5 SE off.
    T, mu, alpha, dt = 10.0, 2.0, 1.0, 0.5 * FS
    bJ, bK, bB = 1.5, 1.5, 1.5
    kT = KB * T
    J, K, B = bJ * kT, bK * kT, bB * kT / (mu * MUB)
    ntri = 256
    side = 2.5
    pos = np.zeros((3 * ntri, 3))
    base = np.arange(ntri) * 20.0
    pos[0::3, 0] = base
    pos[1::3, 0] = base + side
    pos[2::3, 0] = base + 0.5 * side
    pos[2::3, 1] = side * np.sqrt(3.0) / 2.0
    sysd = W.cluster(pos, J=J, rc=3.0, mu=mu, B=(0.0, 0.0, B), T=T, alpha=alpha, dt=dt, K=K, seed=11)
    o = O.Oracle(sysd)
    assert o.ncolours == 3
    v = np.random.default_rng(11).normal(size=(3 * ntri, 3))
    o.set_spins(v / np.linalg.norm(v, axis=1)[:, None])
    b_slow = min(B, 2 * K / (mu * MUB))
    nt = int(round((1 + alpha ** 2) / (alpha * GAMMA * b_slow) / dt))

    def stats(o):
        s = o.spins()
        a, b, c = s[0::3], s[1::3], s[2::3]
        d12, d13, d23 = (a * b).sum(1), (a * c).sum(1), (b * c).sum(1)
        cz = np.stack([a[:, 2], b[:, 2], c[:, 2]], 1)
        e = -bJ * (d12 + d13 + d23) - bK * (cz ** 2).sum(1) - bB * cz.sum(1)
        return np.stack([e, (d12 + d13 + d23) / 3.0, cz.mean(1)], 1)

    per_tri = _time_average(o, 6 * nt, 24, nt // 2, stats)
    m = per_tri.mean(0)
    se = per_tri.std(0, ddof=1) / np.sqrt(ntri)
    want = np.array(_triangle_quadrature((bJ, bJ, bJ), bK, bB))
    assert np.all(np.abs(m - want) < 3 * se), (m, want, se)
