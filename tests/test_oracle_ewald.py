"""Ewald electrostatics of the oracle (coulomb_mode 1): the plain Ewald sum
against the Madelung constant of rock salt, independence of the total
electrostatic energy from the splitting parameter, the smooth-PME sum against
the plain sum, and its gradient against finite differences of its energy."""
import numpy as np
import pytest

from paper_2412_15073_gb300 import systems

C_COUL = 332.0637
MADELUNG_NACL = 1.747564594633   # rock salt, per ion pair, in units of q^2 / r0


def rock_salt(cells, a):
    base = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    na = np.concatenate([base + np.array(c) for c in np.ndindex(cells, cells, cells)]) * a
    cl = na + np.array([0.5, 0, 0]) * a
    x = np.concatenate([na, cl])
    q = np.concatenate([np.ones(len(na)), -np.ones(len(cl))])
    return systems.point_charges(x, cells * a, q, 23.0)


def coulomb_total(o, plain_kmax=None):
    """real-space pairs + reciprocal + self + exclusion terms"""
    e_c = o.energy()[3]                       # real space + smooth-PME part
    if plain_kmax is None:
        return e_c
    _, e_pme, _ = o.ewald_recip_pme()
    _, e_plain = o.ewald_recip_plain(plain_kmax)
    return e_c - e_pme + e_plain


@pytest.mark.parametrize("alpha,kmax", [(0.5, 18), (0.55, 20)])
def test_plain_ewald_gives_the_madelung_energy_of_rock_salt(oracle_mod, alpha, kmax):
    """216 ions of rock salt (a = 5.64 A): the Ewald energy (real space to 8 A,
    the plain reciprocal sum, the self term) is the Madelung energy
    -N/2 C M q^2 / r0, r0 = a/2, to within the truncation of both sums."""
    a = 5.64
    s = rock_salt(3, a)
    o = oracle_mod.Oracle(s, r_cut=8.0, r_split=5.0, dsf_alpha=alpha, coulomb_mode=1, skin=0.2)
    e = coulomb_total(o, plain_kmax=kmax)
    ref = -(s.n / 2) * C_COUL * MADELUNG_NACL / (a / 2)
    assert e == pytest.approx(ref, rel=2e-8)


def test_total_ewald_energy_does_not_depend_on_alpha(oracle_mod, water648):
    es = []
    for alpha in (0.40, 0.45, 0.50):
        o = oracle_mod.Oracle(water648, r_cut=9.0, r_split=5.0, dsf_alpha=alpha, coulomb_mode=1, skin=0.2,
                              skin_outer=0.3)
        es.append(coulomb_total(o, plain_kmax=20))
    # the total is a small difference of large terms (real space about
    # -2300 kcal/mol, self about -18000): 5e-3 kcal/mol is ~3e-7 of them
    assert max(es) - min(es) < 5e-3, es


def test_smooth_pme_matches_the_plain_sum(oracle_mod, water648):
    o = oracle_mod.Oracle(water648, r_cut=9.0, r_split=5.0, dsf_alpha=0.35, coulomb_mode=1, skin=0.2,
                          skin_outer=0.3, pme_order=6, pme_spacing=0.8)
    g_pme, e_pme, K = o.ewald_recip_pme()
    g_plain, e_plain = o.ewald_recip_plain(16)
    assert K >= 24
    assert abs(e_pme - e_plain) < 2e-3          # kcal/mol, with a self term of ~ -15600
    rms = np.sqrt((g_plain ** 2).sum(1).mean())
    assert np.abs(g_pme - g_plain).max() < 1e-3 * rms


def test_smooth_pme_gradient_is_the_derivative_of_its_energy(oracle_mod, water648):
    w = water648.copy()
    p = dict(r_cut=9.0, r_split=5.0, dsf_alpha=0.35, coulomb_mode=1, skin=0.2, skin_outer=0.3, pme_spacing=1.0)
    o = oracle_mod.Oracle(w, **p)
    g, _, _ = o.ewald_recip_pme()
    h = 1e-5
    for i in (0, 1, 300):
        for c in range(3):
            xp = w.x.copy(); xp[i, c] += h
            xm = w.x.copy(); xm[i, c] -= h
            o.set_state(xp, w.v); ep = o.ewald_recip_pme()[1]
            o.set_state(xm, w.v); em = o.ewald_recip_pme()[1]
            assert g[i, c] == pytest.approx((ep - em) / (2 * h), rel=1e-5, abs=1e-6)


def test_ewald_gradient_modes_add_up(oracle_mod, water648):
    """bonded + short + long = full; F0 = bonded + short + reciprocal; mode 6
    is the reciprocal part (with self and exclusion terms)."""
    o = oracle_mod.Oracle(water648, r_cut=9.0, r_split=5.0, dsf_alpha=0.35, coulomb_mode=1, skin=0.2,
                          skin_outer=0.3)
    g = {m: o.gradient(m)[0] for m in range(7)}
    assert np.allclose(g[1] + g[3] + g[4], g[0], atol=1e-9)
    assert np.allclose(g[1] + g[3] + g[6], g[5], atol=1e-9)
    assert np.allclose(g[6], o.ewald_recip_pme()[0], atol=1e-12)


def test_ewald_dynamics_keep_temperature_and_jump_forces_are_weak(oracle_mod, water648):
    """With Ewald electrostatics (alpha 0.35) the pair forces beyond the split
    are small, so the jump range carries little force; BAOAB, JUMP and
    JUMP-RESPA1 (reciprocal part kicked at the outer step) keep 300 K."""
    p = dict(r_cut=9.0, r_split=5.0, h_switch=0.5, dsf_alpha=0.35, coulomb_mode=1, skin=0.2, skin_outer=0.3,
             pme_spacing=1.0)
    o_dsf = oracle_mod.Oracle(water648, r_cut=9.0, r_split=5.0, dsf_alpha=0.2, skin=0.2, skin_outer=0.3)
    o_ew = oracle_mod.Oracle(water648, **p)
    # the long real-space part, |grad|, is an order of magnitude below DSF's
    g_dsf = np.linalg.norm(o_dsf.gradient(4)[0], axis=1).mean()
    g_ew = np.linalg.norm(o_ew.gradient(4)[0] - o_ew.gradient(6)[0], axis=1).mean()
    assert g_ew < 0.2 * g_dsf, (g_ew, g_dsf)
    # from the lattice start the box heats while it relaxes: 40 steps of BAOAB
    # reach nearly the same temperature with Ewald as with DSF (both stand for
    # the same electrostatics); JUMP and JUMP-RESPA1 run without error flags
    kT = 3 * water648.n * 0.0019872042586
    temps = {}
    for name, oo in (("dsf", oracle_mod.Oracle(water648, seed=3, r_cut=9.0, r_split=5.0, dsf_alpha=0.2,
                                                skin=0.2, skin_outer=0.3)),
                     ("ewald", oracle_mod.Oracle(water648, seed=3, **p))):
        assert oo.baoab(40) == 0
        v = oo.state()[1]
        temps[name] = (water648.mass[:, None] * v * v).sum() / 418.4 / kT
    assert abs(temps["ewald"] / temps["dsf"] - 1) < 0.05, temps
    for how, args in (("jump", (40,)), ("jump_respa1", (5, 1.0, 2, 4))):
        o = oracle_mod.Oracle(water648, seed=3, **p)
        assert getattr(o, how)(*args) == 0, how
        assert np.isfinite(o.state()[1]).all()


@pytest.mark.parametrize("order,spacing,tol", [(4, 0.5, 2e-2), (8, 0.8, 5e-4)])
def test_smooth_pme_converges_to_the_plain_sum_for_each_order(oracle_mod, water648, order, spacing, tol):
    """the other B-spline orders the GPU path takes (4 and 8; 6 above)
    interpolate the plain Ewald sum: energy within tol kcal/mol, gradients
    within 1e-3 of their rms"""
    o = oracle_mod.Oracle(water648, r_cut=9.0, r_split=5.0, dsf_alpha=0.35, coulomb_mode=1, skin=0.2,
                          skin_outer=0.3, pme_order=order, pme_spacing=spacing)
    g_pme, e_pme, K = o.ewald_recip_pme()
    g_plain, e_plain = o.ewald_recip_plain(16)
    assert abs(e_pme - e_plain) < tol
    rms = np.sqrt((g_plain ** 2).sum(1).mean())
    assert np.abs(g_pme - g_plain).max() < 1e-3 * rms


def test_smooth_pme_gradient_error_falls_with_the_grid(oracle_mod, water648):
    """refining the grid (order 6) brings the smooth-PME gradient closer to the
    plain sum's: the interpolation error shrinks with the spacing"""
    errs = []
    g_plain = None
    for spacing in (1.2, 0.9, 0.6, 0.5):
        o = oracle_mod.Oracle(water648, r_cut=9.0, r_split=5.0, dsf_alpha=0.35, coulomb_mode=1, skin=0.2,
                              skin_outer=0.3, pme_order=6, pme_spacing=spacing)
        g, _, _ = o.ewald_recip_pme()
        if g_plain is None:
            g_plain, _ = o.ewald_recip_plain(16)
        errs.append(np.abs(g - g_plain).max())
    assert errs[0] > errs[1] > errs[2] > errs[3], errs
    assert errs[0] > 100 * errs[3]


def test_odd_pme_orders_are_refused(oracle_mod, water648):
    """an odd B-spline order makes |b(m)|^2 vanish at m = K/2 on an even grid
    (the Euler exponential spline has a zero at the Nyquist index), so its
    G(m) would divide by zero: only the even orders 4, 6, 8 are taken"""
    with pytest.raises(ValueError):
        oracle_mod.Oracle(water648, r_cut=9.0, coulomb_mode=1, pme_order=5)


EW_EMPTY = dict(r_cut=9.0, r_split=9.6, h_switch=0.5, skin=0.3, seed=4, dsf_alpha=0.35, coulomb_mode=1,
                pme_order=6, pme_spacing=0.8)


def test_jump_mts_equals_baoab_mts_under_ewald_without_jump_range(oracle_mod):
    """Ewald with r_c - h >= r_E: the rings are empty and the (1 - chi) pairs
    vanish, so the outer level of both RESPA1 schemes holds the reciprocal
    part alone: JUMP-RESPA1 reproduces BAOAB-RESPA1 bit for bit. JUMP-RESPA
    kicks the reciprocal part apart from the short pairs that BAOAB-RESPA
    kicks together with it: equal up to rounding."""
    w = systems.water_box(216, box=18.643, seed=0)
    for jump, baoab, args, tol in (("jump_respa1", "baoab_respa1", (4, 1.0, 2, 2), 0.0),
                                   ("jump_respa", "baoab_respa", (6, 1.0, 2), 1e-10)):
        a = oracle_mod.Oracle(w, **EW_EMPTY)
        b = oracle_mod.Oracle(w, **EW_EMPTY)
        getattr(a, jump)(*args)
        getattr(b, baoab)(*args)
        xa, va, _, _ = a.state()
        xb, vb, _, _ = b.state()
        assert np.abs(xa - xb).max() <= tol and np.abs(va - vb).max() <= 10 * tol, jump


def test_baoab_respa1_energy_error_second_order_under_ewald(oracle_mod):
    """At gamma = 0 BAOAB-RESPA1 under Ewald (bonded at delta, short pairs at
    2 delta, the (1 - chi) pairs and the smooth-PME reciprocal part at
    4 delta) is an impulse multiple-time-step Verlet scheme: its total-energy
    fluctuation scales as dt^2. A reciprocal force kicked at the wrong level
    or with the wrong size leaves an error that does not shrink."""
    w = systems.water_box(216, box=18.643, seed=0)
    rms = []
    for dt in (0.2, 0.1):
        o = oracle_mod.Oracle(w, r_cut=9.0, r_split=5.0, h_switch=0.5, gamma=0.0, skin=0.3, dsf_alpha=0.35,
                              coulomb_mode=1, pme_order=6, pme_spacing=0.8)
        outer = 4 * dt
        o.baoab_respa1(int(round(4 / outer)), dt, 2, 2)
        H = []
        for _ in range(int(round(12 / outer))):
            o.baoab_respa1(1, dt, 2, 2)
            _, v, _, _ = o.state()
            ke = 0.5 * (w.mass[:, None] * v * v).sum() / 418.4
            H.append(ke + o.energy().sum())
        rms.append(np.std(H))
    ratio = rms[0] / rms[1]
    assert 3.0 < ratio < 5.0, (rms, ratio)


def test_total_ewald_gradient_is_the_derivative_of_its_energy(oracle_mod, water648):
    """The full gradient under Ewald (bonds, angles, LJ, the real-space
    erfc(alpha r)/r pairs, the smooth-PME reciprocal sum, the self and
    exclusion terms) against central differences of the energy it returns,
    on a few atoms: the real-space derivative has no other pin."""
    w = water648.copy()
    rng = np.random.default_rng(6)
    w.x = (w.x + rng.normal(scale=0.05, size=w.x.shape)) % w.box
    p = dict(r_cut=9.0, r_split=5.0, dsf_alpha=0.35, coulomb_mode=1, skin=0.2, skin_outer=0.3, pme_spacing=1.0)
    o = oracle_mod.Oracle(w, **p)
    g, _ = o.gradient(oracle_mod.GRAD_FULL)
    h = 1e-5
    for i in (0, 1, 2, 301):
        for c in range(3):
            xp = w.x.copy(); xp[i, c] += h
            xm = w.x.copy(); xm[i, c] -= h
            o.set_state(xp, w.v); ep = o.gradient(oracle_mod.GRAD_FULL)[1]
            o.set_state(xm, w.v); em = o.gradient(oracle_mod.GRAD_FULL)[1]
            assert g[i, c] == pytest.approx((ep - em) / (2 * h), rel=1e-5, abs=2e-5)
