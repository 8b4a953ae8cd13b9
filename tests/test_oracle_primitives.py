"""Pins of the oracle's primitives against closed forms, quadrature and
statistics that do not come from the oracle itself.

Sec. 2.2 (rate, Theta, f_eta), Sec. 2.4 (rejection sampling of G~),
Sec. 3.1-3.2 (pair split with chi, bounds), Philox4x32-10 (Salmon et al. 2011).
"""
import math

import numpy as np
import pytest
from scipy import integrate, special, stats

from paper_2412_15073_gb300 import systems

C_COUL = 332.0637


# ---------------------------------------------------------------- Philox
@pytest.mark.parametrize("ctr,key,out", [
    ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
])
def test_philox_known_answers(oracle_mod, ctr, key, out):
    """Philox4x32-10 against the known-answer vectors published with the
    generator (Salmon, Moraes, Dror, Shaw, SC'11: zero, all-ones, and the
    digits of pi as counter and key): the statistics below cannot tell a
    wrong round count or constant from the real thing, these can."""
    assert tuple(int(x) for x in oracle_mod.philox(ctr, key)) == out


def test_philox_uniform_and_independent(oracle_mod):
    """32-bit outputs: flat histogram, decorrelated words, sensitive to every
    counter word and both key words (avalanche)."""
    out = np.array([oracle_mod.philox([i, 7, 3 << 24, 0], [11, 0]) for i in range(20000)],
                   dtype=np.float64)
    u = (out + 0.5) / 2.0 ** 32
    assert abs(u.mean() - 0.5) < 0.005
    assert abs(u.var() - 1 / 12) < 0.002
    h, _ = np.histogram(u.ravel(), bins=64, range=(0, 1))
    chi2 = ((h - h.mean()) ** 2 / h.mean()).sum()
    assert stats.chi2.sf(chi2, 63) > 1e-4
    c = np.corrcoef(u.T)
    assert np.abs(c - np.eye(4)).max() < 0.03
    base = oracle_mod.philox([1, 2, 3, 4], [5, 6])
    for w in range(4):
        ctr = [1, 2, 3, 4]
        ctr[w] ^= 1
        flips = bin(int.from_bytes(np.bitwise_xor(base, oracle_mod.philox(ctr, [5, 6])).tobytes(),
                                   "little")).count("1")
        assert 40 < flips < 88
    for w in range(2):
        key = [5, 6]
        key[w] ^= 1 << 31
        assert not np.array_equal(base, oracle_mod.philox([1, 2, 3, 4], key))


# ---------------------------------------------------------------- Theta
@pytest.mark.parametrize("eta", [-6.0, -3.0, -1.0, -0.2, 0.0, 0.3, 1.0, 2.5, 6.0])
def test_theta_matches_expectation(oracle_mod, eta):
    """Theta(eta) = E[(eta+G)_+] by quadrature of the definition."""
    q, _ = integrate.quad(lambda g: max(eta + g, 0.0) * stats.norm.pdf(g), -eta, np.inf,
                          epsabs=1e-15, epsrel=1e-12)
    assert oracle_mod.theta(eta) == pytest.approx(q, rel=1e-9, abs=1e-14)


def test_theta_identities(oracle_mod):
    """Theta(eta) - Theta(-eta) = eta and Theta'(eta) = Phi(eta)."""
    for eta in np.linspace(-4, 4, 17):
        assert oracle_mod.theta(eta) - oracle_mod.theta(-eta) == pytest.approx(eta, abs=1e-12)
        h = 1e-5
        d = (oracle_mod.theta(eta + h) - oracle_mod.theta(eta - h)) / (2 * h)
        assert d == pytest.approx(stats.norm.cdf(eta), abs=1e-8)


# ---------------------------------------------------------------- G~ sampler
def _ftilde_cdf(y, eta):
    """CDF of f_eta(y) ∝ (eta+y)_+ phi(y)."""
    th = eta * stats.norm.cdf(eta) + stats.norm.pdf(eta)
    y = np.maximum(y, -eta)
    return (eta * (stats.norm.cdf(y) - stats.norm.cdf(-eta)) + stats.norm.pdf(eta)
            - stats.norm.pdf(y)) / th


@pytest.mark.parametrize("eta", [-4.0, -2.5, -1.7, -1.0, -0.4, 0.0, 0.6, 2.0, 5.0])
def test_gtilde_law(oracle_mod, eta):
    """KS test against the exact CDF of f_eta, and E[G~] = Phi(eta)/Theta(eta)."""
    n = 6000
    ys = np.empty(n)
    att = 0
    for k in range(n):
        y, a = oracle_mod.sample_gtilde(eta, seed=3, replica=1, atom=k % 97, s0=k // 97, half=k & 1, k=k)
        assert a > 0
        ys[k] = y
        att += a
    assert (ys >= -eta - 1e-12).all()
    p = stats.kstest(ys, lambda t: _ftilde_cdf(t, eta)).pvalue
    assert p > 1e-4, p
    th = eta * stats.norm.cdf(eta) + stats.norm.pdf(eta)
    mean = stats.norm.cdf(eta) / th
    # variance of G~: E[G~^2] - mean^2 with E[G~^2] = (eta Phi + phi)... use sample sd
    assert abs(ys.mean() - mean) < 5 * ys.std() / math.sqrt(n)
    assert att / n < 3.2


# ---------------------------------------------------------------- pair terms
@pytest.fixture(scope="module")
def pair_sys(oracle_mod):
    w = systems.point_charges(np.array([[0, 0, 0], [6, 0, 0]]), 40.0, [0.5, -0.7], 16.0,
                              lj_eps=0.155, lj_sigma=3.166)
    return oracle_mod.Oracle(w, r_cut=9.0, r_split=5.0, h_switch=0.5, r_mid=5.5, dsf_alpha=0.2)


@pytest.mark.parametrize("weight", [0, 1, 2])
def test_pair_derivative_is_gradient_of_energy(pair_sys, weight):
    """Central differences of the (weighted) pair energy give its radial
    derivative, for LJ + DSF and the chi split."""
    for r in np.concatenate([np.linspace(2.6, 8.95, 60), [4.5, 4.75, 5.0, 5.25]]):
        h = 1e-5
        fd = (pair_sys.pair_u(0, 0, -0.35, r + h, weight) - pair_sys.pair_u(0, 0, -0.35, r - h, weight)) / (2 * h)
        assert pair_sys.pair_dudr(0, 0, -0.35, r, weight) == pytest.approx(fd, rel=2e-7, abs=5e-8)


def test_pair_split_and_cutoff(pair_sys):
    """short + long = full (chi + (1-chi) = 1); DSF and shifted LJ vanish with
    zero slope at r_E; chi = 1 below r_c - h and 0 above r_c."""
    for r in np.linspace(2.5, 10, 200):
        f = pair_sys.pair_dudr(0, 0, 0.3, r, 0)
        s = pair_sys.pair_dudr(0, 0, 0.3, r, 1)
        l = pair_sys.pair_dudr(0, 0, 0.3, r, 2)
        assert s + l == pytest.approx(f, rel=1e-12, abs=1e-13)
        if r <= 4.5:
            assert l == 0.0 and s == f
        if r >= 5.0:
            assert s == 0.0
    R = 9.0
    for w in (0, 2):
        assert abs(pair_sys.pair_u(0, 0, 0.3, R - 1e-9, w)) < 1e-8
        assert abs(pair_sys.pair_dudr(0, 0, 0.3, R - 1e-9, w)) < 1e-8
        assert pair_sys.pair_u(0, 0, 0.3, R + 1e-9, w) == 0.0


def test_dsf_closed_form(pair_sys, oracle_mod):
    """DSF Coulomb (Fennell & Gezelter 2006) at a few radii, written from its
    published definition with scipy's erfc."""
    a, R = 0.2, 9.0
    e0 = oracle_mod.Oracle(systems.point_charges(np.array([[0, 0, 0], [6, 0, 0]]), 40.0, [1.0, 1.0], 16.0),
                           r_cut=R, dsf_alpha=a)
    for r in (1.5, 3.0, 6.0, 8.5):
        ref = C_COUL * (special.erfc(a * r) / r - special.erfc(a * R) / R
                        + (special.erfc(a * R) / R ** 2
                           + 2 * a / math.sqrt(math.pi) * math.exp(-a * a * R * R) / R) * (r - R))
        assert e0.pair_u(0, 0, 1.0, r, 0) == pytest.approx(ref, rel=1e-13)


def test_bounds_dominate_long_gradient(oracle_mod):
    """The ring bounds are >= |d/dr (1-chi) U_DSF| everywhere in their ring
    (checked on a finer, shifted grid and with scipy's bounded minimiser), and
    within 0.5 % of the true maximum."""
    x = np.array([[0, 0, 0], [7, 0, 0], [0, 7, 0]])
    o = oracle_mod.Oracle(systems.point_charges(x, 40.0, [1.0, -1.0, 0.5], 16.0),
                          r_cut=9.0, r_split=5.0, h_switch=0.5, r_mid=5.5, dsf_alpha=0.2)
    lhat, qmax, edges, nr, LY, _ = o.bounds()
    assert nr == 2 and np.allclose(edges, [4.5, 5.5, 9.0])
    f = lambda r: abs(o.pair_dudr(0, 0, 1.0 / C_COUL, r, 2))
    for lo, hi, Lh, Lat in ((4.5, 5.5, lhat[0], LY[0, 0]), (5.5, 9.0, lhat[1], LY[0, 1])):
        rr = np.linspace(lo, hi, 77777)[1:-1] + 1.3e-6
        m = max(f(r) for r in rr)
        opt = __import__("scipy.optimize", fromlist=["x"]).minimize_scalar(
            lambda r: -f(r), bounds=(lo, hi), method="bounded", options={"xatol": 1e-10})
        m = max(m, -opt.fun)
        # the grid max is the true max to 1e-6, and the per-atom bound
        # C |q_i| qmax Lhat (1 + 1e-4), rounded up, dominates the true max
        assert abs(Lh / m - 1) < 1e-6
        exact = C_COUL * 1.0 * qmax * m
        assert exact * (1 + 1e-4) <= Lat <= exact * 1.003
    assert qmax == 1.0


def test_four_ring_bounds_and_lists(oracle_mod, water648):
    """Rings with edges r_c-h, 5.0, 5.5, 7.0, r_E: each ring's bound dominates
    |d/dr (1-chi) U| on its shell, bounds shrink outward, and every partner of
    the two-ring lists appears in the ring lists covering its distance."""
    o = oracle_mod.Oracle(water648, r_cut=9.0, r_split=5.0, h_switch=0.5, skin=0.2, skin_outer=0.3,
                          ring_r=[5.0, 5.5, 7.0])
    lhat, qmax, edges, nr, LY, _ = o.bounds()
    assert nr == 4 and np.allclose(edges, [4.5, 5.0, 5.5, 7.0, 9.0])
    f = lambda r: abs(o.pair_dudr(1, 1, 1.0 / C_COUL, r, 2))   # H-H: Coulomb only
    for y in range(4):
        rr = np.linspace(edges[y], edges[y + 1], 5001)
        assert lhat[y] >= max(f(r) for r in rr) * (1 - 1e-6)
    assert lhat[0] > lhat[1] > lhat[2] > lhat[3]
    two = oracle_mod.Oracle(water648, r_cut=9.0, r_split=5.0, h_switch=0.5, r_mid=5.5, skin=0.2, skin_outer=0.3)
    for i in (0, 1, 200):
        four = set()
        for y in range(4):
            four |= set(o.list_of(y, i).tolist())
        assert set(two.list_of(0, i).tolist()) | set(two.list_of(1, i).tolist()) == four


# ---------------------------------------------------------------- forces
def test_single_molecule_has_no_nonbonded_terms(oracle_mod):
    """Intramolecular pairs are excluded (reading 16): one water alone in
    its box has zero LJ and Coulomb energy and zero nonbonded gradient
    (under DSF), its whole gradient is the bonded one, and the oracle's
    bonded energy is the closed form 1/2 k (r - r0)^2 + 1/2 k_t (t - t0)^2."""
    w = systems.water_box(1, box=24.0, seed=3)
    w.x = w.x + np.random.default_rng(4).normal(scale=0.05, size=w.x.shape)     # strained geometry
    o = oracle_mod.Oracle(w, r_cut=9.0, r_split=5.0, h_switch=0.5, dsf_alpha=0.2, skin=0.3)
    e_bond, e_angle, e_lj, e_coul = o.energy()
    assert e_lj == 0.0 and e_coul == 0.0
    g_nb, _ = o.gradient(oracle_mod.GRAD_NB_FULL)
    assert np.abs(g_nb).max() == 0.0
    g_all, _ = o.gradient(oracle_mod.GRAD_FULL)
    g_b, _ = o.gradient(oracle_mod.GRAD_BONDED)
    np.testing.assert_array_equal(g_all, g_b)
    x = w.x
    ref_b = sum(0.5 * k * (np.linalg.norm(x[i] - x[j]) - r0) ** 2
                for (i, j), k, r0 in zip(w.bonds, w.bond_k, w.bond_r0))
    a, c, b = w.angles[0]
    u, v = x[a] - x[c], x[b] - x[c]
    th = math.acos(u @ v / np.linalg.norm(u) / np.linalg.norm(v))
    ref_a = 0.5 * w.angle_k[0] * (th - w.angle_t0[0]) ** 2
    assert ref_b > 0.1 and ref_a > 1e-3
    assert e_bond == pytest.approx(ref_b, rel=1e-12)
    assert e_angle == pytest.approx(ref_a, rel=1e-12)


def test_total_gradient_finite_differences(oracle_mod, water648):
    """Gradient of the full potential (bonds, angles, LJ, DSF) against central
    differences of the energy, on a few atoms of the 648-atom water box."""
    w = water648.copy()
    rng = np.random.default_rng(5)
    w.x = (w.x + rng.normal(scale=0.05, size=w.x.shape)) % w.box
    o = oracle_mod.Oracle(w, r_cut=9.0)
    g, e = o.gradient(oracle_mod.GRAD_FULL)
    assert e == pytest.approx(o.energy().sum(), rel=1e-12)
    for i in (0, 1, 2, 100, 647):
        for c in range(3):
            h = 1e-5
            xp = w.x.copy(); xp[i, c] += h
            xm = w.x.copy(); xm[i, c] -= h
            o.set_state(xp, w.v); ep = o.energy().sum()
            o.set_state(xm, w.v); em = o.energy().sum()
            assert g[i, c] == pytest.approx((ep - em) / (2 * h), rel=1e-6, abs=1e-6)


def test_gradient_modes_add_up(oracle_mod, water648):
    o = oracle_mod.Oracle(water648, r_cut=9.0)
    full, _ = o.gradient(oracle_mod.GRAD_FULL)
    b, _ = o.gradient(oracle_mod.GRAD_BONDED)
    nb, _ = o.gradient(oracle_mod.GRAD_NB_FULL)
    s, _ = o.gradient(oracle_mod.GRAD_NB_SHORT)
    lg, _ = o.gradient(oracle_mod.GRAD_NB_LONG)
    f0, _ = o.gradient(oracle_mod.GRAD_F0)
    np.testing.assert_allclose(b + nb, full, rtol=1e-12, atol=1e-10)
    np.testing.assert_allclose(s + lg, nb, rtol=1e-12, atol=1e-10)
    np.testing.assert_allclose(b + s, f0, rtol=1e-12, atol=1e-10)
    for i in (3, 77):
        np.testing.assert_allclose(o.gradient_atom(oracle_mod.GRAD_F0, i), f0[i], rtol=1e-12, atol=1e-12)
    # Newton's third law: nonbonded gradients sum to zero
    assert np.abs(nb.sum(0)).max() < 1e-9


# ---------------------------------------------------------------- lists
def test_jump_lists_definition(oracle_mod, water648):
    """Ring lists hold exactly the non-excluded partners with q_i q_j != 0 in
    the skin-widened rings, ordered by (cell of j at the outer rebuild, j) on
    the grid of floor(2 L / (r_E + skin_outer)) cells; checked with numpy."""
    skin = 0.2
    w = water648.copy()
    w.charge = w.charge.copy()
    w.charge[:30] = 0.0                  # ten uncharged molecules: no ring partners (reading 14)
    o = oracle_mod.Oracle(w, r_cut=9.0, r_split=5.0, h_switch=0.5, r_mid=5.5, skin=skin,
                          skin_outer=0.3)
    x = w.x
    L = w.box
    nc = int(math.floor(2 * L / (9.0 + 0.3)))
    cs = L / nc
    cell = np.minimum((x // cs).astype(int), nc - 1)
    lin = (cell[:, 2] * nc + cell[:, 1]) * nc + cell[:, 0]
    mol = np.arange(water648.n) // 3
    rng = np.random.default_rng(0)
    for i in np.concatenate([[0, 1, 2], rng.choice(w.n, 25, replace=False)]):
        d = x[i] - x
        d -= L * np.round(d / L)
        r = np.sqrt((d * d).sum(1))
        ok = (np.arange(w.n) != i) & (mol != mol[i])
        charged = w.charge * w.charge[i] != 0.0
        for kind, lo, hi, extra in ((0, 4.5 - skin, 5.5 + skin, charged),
                                    (1, 5.5 - skin, 9.0 + skin, charged),
                                    (4, 4.5 - skin, 9.0 + skin, w.type == 0)):
            if kind == 4 and w.type[i] != 0:
                extra = np.zeros_like(ok)
            sel = np.flatnonzero(ok & (r >= lo) & (r < hi) & extra)
            sel = sel[np.lexsort((sel, lin[sel]))]
            np.testing.assert_array_equal(o.list_of(kind, i), sel)


def test_lazy_lists_equal_full_lists(oracle_mod, water648):
    """Per-atom lists built on demand (the mode for systems whose O(N^2)
    list build is out of reach) equal the lists built for all atoms, and a
    per-atom C' phase gives the same result in both modes; stepping is
    refused in lazy mode."""
    p = dict(r_cut=9.0, r_split=5.0, h_switch=0.5, skin=0.2, skin_outer=0.3, ring_r=[5.0, 6.0])
    full = oracle_mod.Oracle(water648, **p)
    lazy = oracle_mod.Oracle(water648, lazy_lists=True, **p)
    mt = water648.mass / 418.4
    for i in (0, 1, 2, 300, 647):
        for kind in (0, 1, 2, 3, 4):
            np.testing.assert_array_equal(lazy.list_of(kind, i), full.list_of(kind, i))
        a = -full.gradient_atom(oracle_mod.GRAD_F0, i) / mt[i]
        assert np.array_equal(full.cprime_one(i, water648.v[i], a, 5e-4, 7, 0)[0],
                              lazy.cprime_one(i, water648.v[i], a, 5e-4, 7, 0)[0])
    assert lazy.L.or_step_jump(lazy.h, 1, 1.0) == -1
