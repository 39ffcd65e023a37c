"""Oracle pins: lattice, neighbour lists, exchange function, colouring,
random alloy placement, field and energies -- each checked against an
independent brute-force computation or a value the paper prints."""
import os

import numpy as np
import pytest

import oracle as O
from paper_2608_18541_b300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
MUB = 9.2740100783e-24


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split()
            out[k] = float(v)
    return out


# ---------------------------------------------------------------------------
# Sec. II.E worked example and the 66 % statement
# ---------------------------------------------------------------------------
def test_rederivation_worked_example():
    g = _golden("exchange_rederivation.txt")
    r1 = g["a_fcc"] / np.sqrt(2.0)
    assert abs(r1 - g["r1"]) < 1e-4
    x1, J2, J3 = O.rederive_exchange(r1)
    assert abs(x1 - g["x1"]) < 1e-4
    assert abs(J2 - g["J2"]) < 1e-4
    assert abs(J3 - g["J3"]) < 1e-4
    # the extremum sits at r1 and the value there is J1 (conditions (1), (2))
    assert abs(O.bethe_slater(r1, 1.0, J2, J3) - 1.0) < 1e-12
    assert abs(O.bethe_slater_deriv(r1, 1.0, J2, J3)) < 1e-10


def test_bcc_set_on_fcc_gives_two_thirds():
    g = _golden("exchange_rederivation.txt")
    frac = O.bethe_slater(g["a_fcc"] / np.sqrt(2.0), 1.0, g["bcc_J2"], g["bcc_J3"])
    assert abs(frac - g["fraction_of_J1"]) < 0.01


def test_bethe_slater_derivative_matches_finite_difference():
    for r in (2.0, 2.48, 2.87, 3.3):
        h = 1e-6
        fd = (O.bethe_slater(r + h, 1.7, 0.2171, 1.841) - O.bethe_slater(r - h, 1.7, 0.2171, 1.841)) / (2 * h)
        assert abs(O.bethe_slater_deriv(r, 1.7, 0.2171, 1.841) - fd) < 1e-7 * max(1.0, abs(fd))


# ---------------------------------------------------------------------------
# independent brute force: lattice positions, neighbours, energy
# ---------------------------------------------------------------------------
BASIS = {"sc": [(0, 0, 0)], "bcc": [(0, 0, 0), (.5, .5, .5)],
         "fcc": [(0, 0, 0), (.5, .5, 0), (.5, 0, .5), (0, .5, .5)]}


def _positions(sysd):
    nx, ny, nz, a = sysd["nx"], sysd["ny"], sysd["nz"], sysd["a"]
    pos = []
    for iz in range(nz):
        for iy in range(ny):
            for ix in range(nx):
                for b in BASIS[sysd["lattice"]]:
                    pos.append(((ix + b[0]) * a, (iy + b[1]) * a, (iz + b[2]) * a))
    return np.array(pos), np.array([nx * a, ny * a, nz * a])


def _pair_table(sysd, species):
    """All (i, j, J_ij) with i != j within the cutoff, minimum image, O(N^2)."""
    pos, box = _positions(sysd)
    d = pos[None, :, :] - pos[:, None, :]
    d -= box * np.round(d / box)
    r = np.sqrt((d ** 2).sum(-1))
    n = len(pos)
    Jm = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i == j:
                continue
            e = sysd["exch"][species[i]][species[j]]
            if e["kind"] == "none" or r[i, j] >= e["rc"]:
                continue
            if e["kind"] == "const":
                Jm[i, j] = e["J1"]
            else:
                x = (r[i, j] / e["J3"]) ** 2
                Jm[i, j] = 4 * e["J1"] * x * (1 - e["J2"] * x) * np.exp(-x)
    return Jm


def _energy(sysd, species, Jm, s):
    mu = np.array(sysd["mu"])[species] * MUB
    K = np.array(sysd["K"])[species]
    n_ax = np.array(sysd["axis"])
    B = np.array(sysd["B"])
    e_ex = -0.5 * np.einsum("ij,ik,jk->", Jm, s, s)
    e_an = -(K * (s @ n_ax) ** 2).sum()
    e_z = -(mu * (s @ B)).sum()
    return e_ex, e_an, e_z


def _rand_spins(n, seed):
    r = np.random.default_rng(seed).normal(size=(n, 3))
    return r / np.linalg.norm(r, axis=1, keepdims=True)


SMALL = [
    ("bcc", lambda: W.bcc_fe(3)),
    ("sc_gdfeco", lambda: W.gdfeco_sc(4)),
    ("sc_gdfeco_odd", lambda: W.gdfeco_sc(5)),
]


@pytest.mark.parametrize("name,mk", SMALL)
def test_positions_and_neighbours_match_brute_force(name, mk):
    sysd = mk()
    o = O.Oracle(sysd)
    pos, _ = _positions(sysd)
    assert np.array_equal(o.positions(), pos)
    Jm = _pair_table(sysd, o.species())
    for i in range(o.n):
        j, J = o.neighbours(i)
        ref_j = np.nonzero(Jm[i])[0]
        assert np.array_equal(j, ref_j)            # ascending canonical ids
        assert np.allclose(J, Jm[i, ref_j], rtol=1e-14, atol=0)


@pytest.mark.parametrize("name,mk", SMALL)
def test_field_is_minus_gradient_over_mu(name, mk):
    sysd = mk()
    sysd["B"] = [0.3, -0.2, 1.1]
    o = O.Oracle(sysd)
    spc = o.species()
    Jm = _pair_table(sysd, spc)
    s = _rand_spins(o.n, 3)
    o.set_spins(s)
    for i in (0, 1, o.n // 2, o.n - 1):
        mu = sysd["mu"][spc[i]] * MUB
        grad = np.zeros(3)
        for k in range(3):
            h = 1e-6
            sp, sm = s.copy(), s.copy()
            sp[i, k] += h
            sm[i, k] -= h
            grad[k] = (sum(_energy(sysd, spc, Jm, sp)) - sum(_energy(sysd, spc, Jm, sm))) / (2 * h)
        B = o.field(i)
        assert np.allclose(B, -grad / mu, rtol=1e-6, atol=1e-6 * np.abs(B).max())


@pytest.mark.parametrize("name,mk", SMALL)
def test_observed_energies_and_magnetisation(name, mk):
    sysd = mk()
    sysd["B"] = [0.0, 0.4, 2.0]
    o = O.Oracle(sysd)
    spc = o.species()
    Jm = _pair_table(sysd, spc)
    s = _rand_spins(o.n, 5)
    o.set_spins(s)
    obs = o.observe()
    e_ex, e_an, e_z = _energy(sysd, spc, Jm, s)
    assert np.isclose(obs[10], e_ex, rtol=1e-12, atol=0)
    assert np.isclose(obs[11], e_an, rtol=1e-12, atol=0)
    assert np.isclose(obs[12], e_z, rtol=1e-12, atol=0)
    for t in range(sysd["nspecies"]):
        assert np.allclose(obs[1 + 3 * t:4 + 3 * t], s[spc == t].mean(0), rtol=0, atol=1e-14)
    mu = np.array(sysd["mu"])[spc]
    assert np.allclose(obs[7:10], (mu[:, None] * s).sum(0) / mu.sum(), atol=1e-14)


# ---------------------------------------------------------------------------
# colouring
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("mk,K", [
    (lambda: W.bcc_fe(4), 4),          # bcc NN+NNN, even L: 2 * basis + parity
    (lambda: W.gdfeco_sc(6), 2),       # sc NN, even L: parity
    (lambda: W.gdfeco_sc(5), 3),       # sc NN, odd L: not bipartite -> mod-3 rule
    (lambda: W.gdfeco_sc(7), 3),
    (lambda: W.gdfeco_sc(13), 3),
    (lambda: W.gdfeco_sc(9), 3),
    (lambda: W.single_spins(8), 1),    # no coupling at all: one colour
])
def test_colouring_is_proper_and_minimal_where_known(mk, K):
    sysd = mk()
    o = O.Oracle(sysd)
    col = o.colours()
    assert o.ncolours == K
    assert col.min() == 0 and col.max() == K - 1
    if sysd["exch"][0][0]["kind"] != "none":
        Jm = _pair_table(sysd, o.species())
        ii, jj = np.nonzero(Jm)
        assert not np.any(col[ii] == col[jj])


def test_greedy_fallback_on_odd_bcc():
    # the bcc rule 2 * basis + parity breaks across the wrap of an odd box; the
    # greedy colouring that replaces it must still be proper
    sysd = W.bcc_fe(5)
    o = O.Oracle(sysd)
    col = o.colours()
    Jm = _pair_table(sysd, o.species())
    ii, jj = np.nonzero(Jm)
    assert not np.any(col[ii] == col[jj])
    assert o.ncolours >= 4
    # greedy in ascending id: atom 0 takes colour 0, and every atom's colour is the
    # smallest one absent from its lower-id neighbours
    assert col[0] == 0
    for i in range(o.n):
        lower = {col[j] for j in np.nonzero(Jm[i])[0] if j < i}
        assert col[i] == min(set(range(o.ncolours + 1)) - lower)


def test_fcc_basis_colouring():
    sysd = W.bcc_fe(4)
    sysd["lattice"] = "fcc"
    sysd["a"] = 3.6
    sysd["exch"] = [[{"kind": "const", "J1": 1e-21, "rc": 3.0}]]
    o = O.Oracle(sysd)
    assert o.ncolours == 4
    assert np.array_equal(o.colours(), np.arange(o.n) % 4)


# ---------------------------------------------------------------------------
# random alloy placement (Sec. II.D)
# ---------------------------------------------------------------------------
def test_placement_exact_count_and_uniform_marginal():
    sysd = W.gdfeco_sc(6)
    n = 216
    R = 300
    counts = np.zeros(n)
    prev = None
    for r in range(R):
        sp = O.Oracle(sysd, instance=r).species()
        assert sp.sum() == 54                    # round(0.25 * 216)
        counts += sp
        if prev is not None:
            assert not np.array_equal(prev, sp)   # a fresh alloy per realisation
        prev = sp
    # each site is Gd with probability 1/4: binomial(R, 1/4) per site
    sd = np.sqrt(R * 0.25 * 0.75)
    assert np.all(np.abs(counts - R * 0.25) < 5 * sd)
    chi2 = ((counts - R * 0.25) ** 2 / (R * 0.25 * 0.75)).sum()
    assert chi2 < n + 6 * np.sqrt(2 * n)
    # reproducible
    assert np.array_equal(O.Oracle(sysd, instance=3).species(), O.Oracle(sysd, instance=3).species())


def test_placement_rounding_of_count():
    sysd = W.gdfeco_sc(5)            # 125 sites
    for frac, expect in ((0.25, 31), (0.2, 25), (0.3, 38), (0.0, 0)):
        sysd["frac1"] = frac
        assert O.Oracle(sysd).species().sum() == expect


def test_box_must_exceed_twice_cutoff():
    sysd = W.bcc_fe(2)   # 5.73 A box vs 3.5 A cutoff
    with pytest.raises(ValueError):
        O.Oracle(sysd)
