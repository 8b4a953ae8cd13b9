"""Pins of the oracle's integrators and jump processes against laws that hold
independently of the oracle: thinning survival laws (Sec. 2.4, exactness of
Poisson thinning), the BPS bounce law (Sec. 2.2/3.2), invariance of the Gibbs
measure (Sec. 2.2, the jump mechanism leaves mu invariant), exact harmonic
configurational sampling of BAOAB (Leimkuhler & Matthews 2013), second order
of velocity Verlet, and reductions between integrators (Sec. 2.3).
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats

from paper_2412_15073_gb300 import systems

KB = 0.0019872042586
KCAL_AMU = 418.4
C_COUL = 332.0637


def beta_of(T=300.0):
    return 1.0 / (KB * T)


# ------------------------------------------------------------ thinning laws
def _ring_system(oracle_mod, eps_mode=1, eps0=0.1, ring_r=None):
    """Atom 0 with four charged partners in the jump rings (4.8, 5.2, 6.0, 8.0 A)."""
    x = np.array([[10, 10, 10], [14.8, 10, 10], [10, 15.2, 10], [10, 10, 16.0], [4.34, 15.66, 10]])
    w = systems.point_charges(x, 30.0, [0.5, -0.7, 0.4, -0.3, 0.6], [16.0, 1, 1, 1, 1])
    return oracle_mod.Oracle(w, r_cut=9.0, r_split=5.0, h_switch=0.5, r_mid=5.5, dsf_alpha=0.2,
                             skin=0.3, eps0=eps0, eps_mode=eps_mode, seed=21, ring_r=ring_r)


def _pair_rates(o, v, eps_mode, eps0, beta, mt):
    """sum_j lambda_ij(v) from the paper's per-pair rate (Sec. 3.1),
    lambda = sqrt(beta)/(eps sqrt(m)) |F| Theta(eps sqrt(beta m) v.F/|F|), with
    eps = eps0 |F| (adaptive) or eps0 (constant); F from the pinned pair
    derivative of the long part."""
    x, _, _, _ = o.state()
    tot = 0.0
    q = [0.5, -0.7, 0.4, -0.3, 0.6]
    for j in range(1, 5):
        d = x[0] - x[j]
        r = np.linalg.norm(d)
        F = o.pair_dudr(0, 0, q[0] * q[j], r, 2) * d / r
        Fn = np.linalg.norm(F)
        if Fn == 0:
            continue
        eps = eps0 * Fn if eps_mode == 1 else eps0
        eta = eps * math.sqrt(beta * mt) * (v @ F) / Fn
        th = eta * stats.norm.cdf(eta) + stats.norm.pdf(eta)
        tot += math.sqrt(beta) / (eps * math.sqrt(mt)) * Fn * th
    return tot


@pytest.mark.parametrize("eps_mode,rings", [(1, None), (0, None), (1, [5.0, 5.5, 7.0]), (0, [5.0, 7.0])])
def test_cprime_first_jump_survival_a0(oracle_mod, eps_mode, rings):
    """With a = 0 the accepted jumps of the first event form a Poisson process
    of rate sum_j lambda_ij(v): P(no jump in tau/2) = exp(-tau/2 sum lambda),
    whatever the ring partition of the bound (two rings, or three and four)."""
    eps0 = 0.1 if eps_mode == 1 else 2.0
    o = _ring_system(oracle_mod, eps_mode, eps0, rings)
    beta, mt = beta_of(), 16.0 / KCAL_AMU
    v = np.array([3.0, -2.0, 4.0])
    lam = _pair_rates(o, v, eps_mode, eps0, beta, mt)
    tau2 = 1.0 / lam
    n = 20000
    none = 0
    props = 0
    for s0 in range(n):
        vo, npr, na = o.cprime_one(0, v, np.zeros(3), tau2, s0, 0)
        none += na == 0
        props += npr
    p_exp = math.exp(-tau2 * lam)
    se = math.sqrt(p_exp * (1 - p_exp) / n)
    assert abs(none / n - p_exp) < 4.5 * se, (none / n, p_exp)
    assert o.errors == 0
    assert props / n > lam * tau2   # a proper bound proposes more than it accepts


@pytest.mark.parametrize("a", [(-900.0, 1400.0, 600.0), (2700.0, -1400.0, 1800.0)])
def test_cprime_first_jump_survival_with_drift(oracle_mod, a):
    """With a != 0, v(s) = v + s a until the first jump, so
    P(no jump in tau/2) = exp(-int_0^{tau/2} sum_j lambda_ij(v + s a) ds).
    The drift slows the atom down first (v.a < 0) or speeds it up (v.a > 0,
    where the bound on |v| must hold the s^2 |a|^2 term: no ratio above 1)."""
    o = _ring_system(oracle_mod)
    beta, mt = beta_of(), 16.0 / KCAL_AMU
    v = np.array([2.0, -1.0, 1.0])
    a = np.array(a)
    lam0 = _pair_rates(o, v, 1, 0.1, beta, mt)
    tau2 = 1.2 / lam0
    integ, _ = integrate.quad(lambda s: _pair_rates(o, v + s * a, 1, 0.1, beta, mt), 0, tau2)
    n = 20000
    none = 0
    for s0 in range(n):
        vo, npr, na = o.cprime_one(0, v, a, tau2, s0, 1)
        none += na == 0
        if na == 0:   # no jump: v ends exactly at v + tau/2 a
            np.testing.assert_allclose(vo, v + tau2 * a, rtol=1e-12, atol=1e-12)
    p_exp = math.exp(-integ)
    se = math.sqrt(p_exp * (1 - p_exp) / n)
    assert abs(none / n - p_exp) < 4.5 * se, (none / n, p_exp)
    assert o.errors == 0


def test_jprime_single_bounce_law(oracle_mod):
    """BPS on one LJ pair with v.F > 0: at most one reflection, with
    probability 1 - exp(-beta (v.F)_+ tau/2); |v| is preserved (Sec. 3.2)."""
    x = np.array([[10, 10, 10], [16.2, 10, 10]])
    w = systems.point_charges(x, 30.0, [0.0, 0.0], 16.0, lj_eps=0.155, lj_sigma=3.166)
    o = oracle_mod.Oracle(w, r_cut=9.0, r_split=5.0, h_switch=0.5, skin=0.3, seed=5)
    r = 6.2
    F = o.pair_dudr(0, 0, 0.0, r, 2) * np.array([-1.0, 0, 0])    # grad_x0 of (1-chi)U_LJ
    v = np.array([-4.0, 1.0, 0.5]) * (1 if F[0] < 0 else -1)
    vF = v @ F
    assert vF > 0
    beta = beta_of()
    tau2 = 0.7 / (beta * vF)
    n = 20000
    bounced = 0
    for s0 in range(n):
        vo, npr, na = o.jprime_one(0, v, tau2, s0, 0)
        assert na <= 1
        bounced += na
        assert np.linalg.norm(vo) == pytest.approx(np.linalg.norm(v), rel=1e-14)
        if na:
            np.testing.assert_allclose(vo, v - 2 * vF / (F @ F) * F, rtol=1e-12)
    p_exp = 1 - math.exp(-beta * vF * tau2)
    se = math.sqrt(p_exp * (1 - p_exp) / n)
    assert abs(bounced / n - p_exp) < 4.5 * se


# ------------------------------------------------------------ invariance
@pytest.mark.slow
@pytest.mark.parametrize("eps_mode,eps0", [(1, 0.1), (0, 2.0)])
def test_jump_samples_boltzmann_two_body(oracle_mod, eps_mode, eps0):
    """JUMP (C'J'AOAJ'C') on two charged LJ atoms: the pair distance follows
    r^2 exp(-beta U(r)) (Gibbs invariance, Sec. 2.2), where U includes the
    long-range part that only the jumps carry. The same data must reject the
    law of the short part alone, which shows the jumps matter. Adaptive eps
    (small here) and a large constant eps, where the 1 + eps^2 of the jump
    size matters."""
    oracle_mod.set_threads(1)
    L = 12.0
    beta = beta_of()
    edges = np.linspace(2.6, 6.0, 18)
    hists = []
    o = None
    for chain in range(8):
        w = systems.point_charges(np.array([[1, 1, 1], [5, 1, 1]]), L, [0.2, -0.2], 4.0,
                                  lj_eps=0.2, lj_sigma=3.0, seed=chain)
        o = oracle_mod.Oracle(w, r_cut=5.5, r_split=3.5, h_switch=0.5, r_mid=4.2, dsf_alpha=0.2,
                              gamma=5.0, skin=0.4, eps0=eps0, eps_mode=eps_mode, seed=100 + chain)
        rs = []
        for it in range(25100):
            o.jump(20)
            x, v, _, _ = o.state()
            # a wrong jump size heats the pair without bound: fail at once
            ke_T = 4.0 * (v * v).sum() / KCAL_AMU / (6 * KB)
            assert o.errors == 0 and ke_T < 5000.0, (chain, it, ke_T)
            if it < 100:
                continue                                    # 2000 steps of burn-in
            d = x[0] - x[1]
            d -= L * np.round(d / L)
            rs.append(math.sqrt(d @ d))
        rs = np.array(rs)
        rs = rs[rs < 6.0]
        h, _ = np.histogram(rs, bins=edges)
        hists.append(h / len(rs))
        assert o.errors == 0
    oracle_mod.set_threads(0)
    hists = np.array(hists)
    mean, se = hists.mean(0), hists.std(0, ddof=1) / math.sqrt(len(hists))

    def law(weight):
        pr = lambda r: r * r * math.exp(-beta * o.pair_u(0, 0, -0.04, r, weight))
        Z = integrate.quad(pr, 0.5, 6.0, limit=200)[0]
        return np.array([integrate.quad(pr, a, b)[0] / Z for a, b in zip(edges[:-1], edges[1:])])

    z_full = (mean - law(0)) / se
    z_short = (mean - law(1)) / se
    assert np.abs(z_full).max() < 5.0, z_full
    assert np.abs(z_short).max() > 15.0


def _harmonic_chain(seed):
    """Four atoms bonded in a chain 0-1-2-3 (no angles, no exclusions).
    Atoms 0 and 1 carry charges +-0.3 and LJ (eps 0.8, sigma 3.0), so the pair
    (0, 1) is bonded and also interacts through LJ + DSF; atoms 2 and 3 have no
    nonbonded terms. The Gibbs density then factorises over the three bond
    vectors: bond 0-1 has the length law r^2 exp(-beta (k/2 (r - 4.2)^2 + U(r))),
    bonds 1-2 and 2-3 that of a free harmonic spring, r^2 exp(-beta k/2 (r - 3)^2)."""
    x = np.array([[2.0, 7.0, 7.0], [6.2, 7.0, 7.0], [9.2, 7.0, 7.0], [12.2, 7.0, 7.0]])
    w = systems.point_charges(x, 14.0, [0.3, -0.3, 0.0, 0.0], 4.0, seed=seed)
    w.type = np.array([0, 0, 1, 1], dtype=np.int32)
    w.lj_eps = np.array([[0.8, 0.0], [0.0, 0.0]])
    w.lj_sigma = np.array([[3.0, 1.0], [1.0, 1.0]])
    w.bonds = np.array([[0, 1], [1, 2], [2, 3]], dtype=np.int32)
    w.bond_k = np.array([3.0, 3.0, 3.0])
    w.bond_r0 = np.array([4.2, 3.0, 3.0])
    return w


@pytest.mark.slow
@pytest.mark.parametrize("integ,lj_long_mode", [("jump", 0), ("jump_respa", 0), ("jump_respa1", 0),
                                                ("jump_respa1", 2)])
def test_multiple_time_step_jumps_sample_boltzmann_harmonic_chain(oracle_mod, integ, lj_long_mode):
    """Gibbs invariance (Sec. 2.2) of the JUMP family with its multiple time
    steps (Sec. 2.3) on a harmonic chain: bonds in F0 at the inner step delta,
    the short pair part and the pair jumps at Delta = 2 delta (JUMP-RESPA) or
    at kappa = 2 delta with an outer level at 2 kappa (JUMP-RESPA1; with
    lj_long_mode 2 that level kicks the (1 - chi) LJ part). The three bond
    lengths must follow their exact laws (the long-range pair part of bond
    0-1 is carried by the jumps alone); the law of the short pair part alone
    must be rejected. Bin z-scores use one variance inflation factor for the
    correlation of the samples, pooled over the bins of a bond."""
    oracle_mod.set_threads(1)
    beta = beta_of()
    L = 14.0
    p = dict(r_cut=5.5, r_split=3.6, h_switch=0.5, r_mid=4.4, dsf_alpha=0.2, gamma=5.0, skin=0.4,
             eps0=0.1, eps_mode=1, lj_long_mode=lj_long_mode)
    run = {"jump": lambda o: o.jump(20), "jump_respa": lambda o: o.jump_respa(10, 1.0, 2),
           "jump_respa1": lambda o: o.jump_respa1(5, 1.0, 2, 2)}[integ]
    edges = [np.linspace(2.8, 6.0, 17), np.linspace(1.6, 4.4, 15), np.linspace(1.6, 4.4, 15)]
    bonds = ((0, 1), (1, 2), (2, 3))
    hists = [[], [], []]
    o = None
    for chain in range(16):
        o = oracle_mod.Oracle(_harmonic_chain(chain), seed=200 + chain, **p)
        rs = []
        for it in range(6500):
            run(o)                                          # 20 fs
            assert o.errors == 0, (chain, it)
            if it < 100:
                continue                                    # 2 ps of burn-in
            x = o.state()[0]
            row = []
            for a, b in bonds:
                d = x[a] - x[b]
                d -= L * np.round(d / L)
                row.append(math.sqrt(d @ d))
            rs.append(row)
        rs = np.array(rs)
        for k in range(3):
            h, _ = np.histogram(rs[:, k], bins=edges[k])
            hists[k].append(h / len(rs))
    oracle_mod.set_threads(0)

    def law(u, e):
        pr = lambda r: r * r * math.exp(-beta * u(r))
        Z = integrate.quad(pr, 0.5, 6.9, limit=200)[0]
        return np.array([integrate.quad(pr, a, b)[0] / Z for a, b in zip(e[:-1], e[1:])])

    def zscores(h, pb):
        h = np.asarray(h)
        use = pb > 0.01
        tau = np.mean(h[:, use].var(0, ddof=1) / (pb[use] * (1 - pb[use])))
        return np.where(use, (h.mean(0) - pb) / np.sqrt(tau * pb * (1 - pb) / len(h)), 0.0)

    full = lambda r: 1.5 * (r - 4.2) ** 2 + o.pair_u(0, 0, -0.09, r, 0)
    short = lambda r: 1.5 * (r - 4.2) ** 2 + o.pair_u(0, 0, -0.09, r, 1)
    spring = lambda r: 1.5 * (r - 3.0) ** 2
    z01 = zscores(hists[0], law(full, edges[0]))
    assert np.abs(z01).max() < 5.0, z01
    for k in (1, 2):
        zk = zscores(hists[k], law(spring, edges[k]))
        assert np.abs(zk).max() < 5.0, (k, zk)
    assert np.abs(zscores(hists[0], law(short, edges[0]))).max() > 10.0


# ------------------------------------------------------------ BAOAB
def test_baoab_exact_harmonic_configurations(oracle_mod):
    """BAOAB samples the configurational law of a harmonic oscillator exactly
    for any stable step (Leimkuhler & Matthews 2013): var(d) = kT/k per axis
    for U = k/2 |x0 - x1|^2, here at omega dt = 1.45."""
    oracle_mod.set_threads(1)
    k = 100.0
    w = systems.point_charges(np.array([[5, 5, 5], [5.05, 5, 5]]), 30.0, [0.0, 0.0], 1.0)
    w.bonds = np.array([[0, 1]], dtype=np.int32)
    w.bond_k = np.array([k])
    w.bond_r0 = np.array([0.0])
    w.excl = np.array([[0, 1]], dtype=np.int32)
    var = []
    for chain in range(4):
        o = oracle_mod.Oracle(w, r_cut=9.0, gamma=20.0, skin=2.0, seed=chain)
        o.baoab(500, dt_fs=5.0)
        ds = []
        for _ in range(20000):
            o.baoab(5, dt_fs=5.0)
            x = o.state()[0]
            d = x[0] - x[1]
            ds.append(d - 30.0 * np.round(d / 30.0))
        var.append(np.var(np.array(ds)))
    oracle_mod.set_threads(0)
    target = KB * 300.0 / k
    assert abs(np.mean(var) / target - 1) < 0.02, np.array(var) / target


def test_verlet_energy_error_second_order(oracle_mod, water648):
    """At gamma = 0 BAOAB is velocity Verlet: the RMS fluctuation of the total
    energy scales as dt^2 (ratio ~ 4 when dt halves)."""
    rms = []
    for dt in (0.4, 0.2):
        o = oracle_mod.Oracle(water648, r_cut=9.0, gamma=0.0, skin=0.3)
        o.baoab(int(round(4 / dt)), dt_fs=dt)     # let the lattice start settle a little
        H = []
        for _ in range(int(round(16 / dt))):
            o.baoab(1, dt_fs=dt)
            _, v, _, _ = o.state()
            ke = 0.5 * (water648.mass[:, None] * v * v).sum() / KCAL_AMU
            H.append(ke + o.energy().sum())
        rms.append(np.std(H))
    ratio = rms[0] / rms[1]
    assert 3.0 < ratio < 5.0, (rms, ratio)


@pytest.mark.parametrize("integ,per_outer", [("baoab_respa", 2), ("baoab_respa1", 4)])
def test_multiple_time_step_energy_error_second_order(oracle_mod, water648, integ, per_outer):
    """At gamma = 0 BAOAB-RESPA (bonded at delta, nonbonded at 2 delta) and
    BAOAB-RESPA1 (bonded at delta, short pairs at 2 delta, long pairs at
    4 delta) are impulse multiple-time-step Verlet schemes (Sec. 2.3): the
    RMS fluctuation of the total energy at the outer steps scales as dt^2
    (ratio ~ 4 when every step halves). A kick of the wrong size at any level
    leaves an error that does not shrink with dt."""
    rms = []
    for dt in (0.2, 0.1):
        o = oracle_mod.Oracle(water648, r_cut=9.0, gamma=0.0, skin=0.3)
        step = (lambda k: o.baoab_respa(k, dt, 2)) if integ == "baoab_respa" else \
            (lambda k: o.baoab_respa1(k, dt, 2, 2))
        outer = dt * per_outer
        step(int(round(4 / outer)))
        H = []
        for _ in range(int(round(16 / outer))):
            step(1)
            _, v, _, _ = o.state()
            ke = 0.5 * (water648.mass[:, None] * v * v).sum() / KCAL_AMU
            H.append(ke + o.energy().sum())
        rms.append(np.std(H))
    ratio = rms[0] / rms[1]
    assert 3.0 < ratio < 5.0, (rms, ratio)


# ------------------------------------------------------------ reductions
def test_jump_equals_baoab_without_jump_range(oracle_mod, water648):
    """r_c - h >= r_E: chi = 1 on all pairs, the rings are empty, C' is the B
    kick and J' does nothing; JUMP reproduces BAOAB bit for bit."""
    a = oracle_mod.Oracle(water648, r_cut=9.0, r_split=9.6, h_switch=0.5, skin=0.3, seed=4)
    b = oracle_mod.Oracle(water648, r_cut=9.0, r_split=9.6, h_switch=0.5, skin=0.3, seed=4)
    assert a.list_counts(0).sum() == 0 and a.list_counts(1).sum() == 0 and a.list_counts(2).sum() == 0
    a.jump(30)
    b.baoab(30)
    xa, va, _, _ = a.state()
    xb, vb, _, _ = b.state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)


@pytest.mark.parametrize("jump,baoab,args", [("jump_respa", "baoab_respa", (15, 1.0, 2)),
                                             ("jump_respa1", "baoab_respa1", (8, 1.0, 2, 2))])
def test_jump_mts_equals_baoab_mts_without_jump_range(oracle_mod, water648, jump, baoab, args):
    """r_c - h >= r_E: the rings are empty, C' is the B kick of the short
    (here the whole) nonbonded force and the long level is empty under DSF:
    JUMP-RESPA and JUMP-RESPA1 reproduce BAOAB-RESPA and BAOAB-RESPA1 bit for
    bit, so their multiple-time-step skeletons are those the energy test
    above pins."""
    p = dict(r_cut=9.0, r_split=9.6, h_switch=0.5, skin=0.3, seed=4)
    a = oracle_mod.Oracle(water648, **p)
    b = oracle_mod.Oracle(water648, **p)
    getattr(a, jump)(*args)
    getattr(b, baoab)(*args)
    xa, va, _, _ = a.state()
    xb, vb, _, _ = b.state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    assert a.step == b.step


def test_respa_one_inner_step_is_baoab(oracle_mod, water648):
    """BAOAB-RESPA with n = 1 and BAOAB-RESPA1 with m = n = 1 are BAOAB, up to
    the order in which the bonded and nonbonded kicks are added."""
    ref = oracle_mod.Oracle(water648, r_cut=9.0, skin=0.3, seed=2)
    ref.baoab(20)
    xr, vr, _, _ = ref.state()
    for how in ("respa", "respa1"):
        o = oracle_mod.Oracle(water648, r_cut=9.0, skin=0.3, seed=2)
        if how == "respa":
            o.baoab_respa(20, 1.0, 1)
        else:
            o.baoab_respa1(20, 1.0, 1, 1)
        x, v, _, _ = o.state()
        assert np.abs(x - xr).max() < 1e-10
        assert np.abs(v - vr).max() < 1e-8


def test_jump_respa1_is_jump_respa_at_mid_level(oracle_mod, water648):
    """Without a slow many-body force the JUMP-RESPA1 outer level is empty:
    n_outer x n mid cycles of m inner steps equal JUMP-RESPA with n_inner = m."""
    a = oracle_mod.Oracle(water648, r_cut=9.0, skin=0.3, seed=8)
    b = oracle_mod.Oracle(water648, r_cut=9.0, skin=0.3, seed=8)
    a.jump_respa1(3, 1.0, 2, 2)
    b.jump_respa(6, 1.0, 2)
    assert a.step == b.step == 12
    xa, va, _, _ = a.state()
    xb, vb, _, _ = b.state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)


def test_jump_respa_one_inner_step_matches_jump_statistics(oracle_mod, water648):
    """JUMP-RESPA with n_inner = 1 moves bonded forces from the C' drift into
    B kicks; both keep the water box at the bath temperature over 200 fs and
    run without bound violations."""
    for how in ("jump", "respa"):
        o = oracle_mod.Oracle(water648, r_cut=9.0, skin=0.3, seed=3)
        o.jump(200) if how == "jump" else o.jump_respa(200, 1.0, 1)
        assert o.errors == 0
        _, v, _, _ = o.state()
        T = (water648.mass[:, None] * v * v).sum() / KCAL_AMU / (3 * water648.n * KB)
        assert 250 < T < 350


def test_resume_is_bit_exact(oracle_mod, water648):
    """Counter-based streams: 2k steps equal k steps, a save/restore of
    (x, v, images, list-build and outer-rebuild positions, step), then k more."""
    a = oracle_mod.Oracle(water648, r_cut=9.0, skin=0.2, skin_outer=0.3, seed=6)
    a.jump(40)
    xa, va, _, _ = a.state()
    b = oracle_mod.Oracle(water648, r_cut=9.0, skin=0.2, skin_outer=0.3, seed=6)
    b.jump(20)
    x, v, img, xb, xo = b.state(outer=True)
    c = oracle_mod.Oracle(water648, r_cut=9.0, skin=0.2, skin_outer=0.3, seed=6)
    c.set_state(x, v, img, xb, step=20, x_outer=xo)
    c.jump(20)
    xc, vc, _, _ = c.state()
    assert np.array_equal(xa, xc) and np.array_equal(va, vc)


def test_event_log_and_rate_bound_hold_on_water(oracle_mod, water648):
    """100 JUMP steps on 648 waters: no bound violation (p <= 1 always), an
    event log that agrees with the counters, and sane jump statistics."""
    o = oracle_mod.Oracle(water648, r_cut=9.0, skin=0.3, seed=1)
    o.events_enable(1 << 22)
    o.jump(100)
    assert o.errors == 0
    c = o.counters()
    ev = o.events()
    assert len(ev) == c[1] + c[3]
    assert (ev[:, 2] == 2).sum() == c[1] and (ev[:, 2] == 3).sum() == c[3]
    per_atom_step = c[0] / (648 * 100)
    assert 20 < per_atom_step < 120
    assert 0.05 < c[1] / c[0] < 0.6


def test_lj_long_mode_moves_the_lj_long_part_into_f0(oracle_mod, water648):
    """With the LJ long part deterministic (the paper's GPU runs), the short
    gradient gains exactly what the long one loses, the total is unchanged,
    the moved part is the (1-chi) LJ gradient alone, and JUMP proposes no
    LJ bounces."""
    w = water648.copy()
    w.x = (w.x + np.random.default_rng(2).normal(scale=0.05, size=w.x.shape)) % w.box
    p = dict(r_cut=9.0, r_split=5.0, h_switch=0.5, skin=0.2, skin_outer=0.3)
    a = oracle_mod.Oracle(w, **p)
    b = oracle_mod.Oracle(w, lj_long_mode=1, **p)
    g = {(o, m): o.gradient(m)[0] for o in (a, b) for m in (0, 3, 4, 5)}
    assert np.allclose(g[(a, 0)], g[(b, 0)], rtol=0, atol=1e-12)
    moved = g[(b, 3)] - g[(a, 3)]
    assert np.allclose(moved, g[(a, 4)] - g[(b, 4)], rtol=0, atol=1e-10)
    assert np.allclose(g[(b, 5)] - g[(a, 5)], moved, rtol=0, atol=1e-10)
    # the moved part: (1-chi) LJ summed over O-O pairs (water has LJ on O only)
    oxy = np.flatnonzero(w.type == 0)
    i = int(oxy[3])
    ref = np.zeros(3)
    for j in oxy:
        if j == i or j // 3 == i // 3:
            continue
        d = w.x[i] - w.x[j]
        d -= w.box * np.round(d / w.box)
        r = np.linalg.norm(d)
        if r < 9.0:
            ref += a.pair_dudr(0, 0, 0.0, r, 2) * d / r
    assert np.allclose(moved[i], ref, rtol=1e-10, atol=1e-12)
    b.jump(5)
    assert b.counters()[2] == 0 and b.counters()[0] > 0


def test_lj_long_mode_2_holds_the_lj_long_part_at_the_slow_level(oracle_mod, water648):
    """lj_long_mode 2: modes 3 and 4 are those of mode 0 (LJ split by chi),
    mode 6 is the (1-chi) LJ gradient that mode 1 moved into the short part,
    F0 (mode 5) is that of mode 1, no LJ bounces; JUMP-RESPA1 (which kicks
    the slow part at its outer step) runs without bounces or errors."""
    w = water648.copy()
    w.x = (w.x + np.random.default_rng(2).normal(scale=0.05, size=w.x.shape)) % w.box
    p = dict(r_cut=9.0, r_split=5.0, h_switch=0.5, skin=0.2, skin_outer=0.3)
    a = oracle_mod.Oracle(w, **p)
    b = oracle_mod.Oracle(w, lj_long_mode=1, **p)
    c = oracle_mod.Oracle(w, lj_long_mode=2, **p)
    ga = {m: a.gradient(m)[0] for m in (0, 3, 4, 5, 6)}
    gb = {m: b.gradient(m)[0] for m in (0, 3, 4, 5, 6)}
    gc = {m: c.gradient(m)[0] for m in (0, 1, 3, 4, 5, 6)}
    for m in (0, 3, 4):
        assert np.array_equal(gc[m], ga[m]), m
    assert np.allclose(gc[5], gb[5], rtol=0, atol=1e-10)
    assert np.allclose(gc[6], gb[3] - ga[3], rtol=0, atol=1e-10)       # the (1-chi) LJ part
    assert np.allclose(gc[1] + gc[3] + gc[6], gc[5], rtol=0, atol=1e-10)
    assert not ga[6].any() and not gb[6].any()
    # per atom, as the atom-wise call computes it
    i = int(np.flatnonzero(w.type == 0)[5])
    np.testing.assert_allclose(c.gradient_atom(6, i), gc[6][i], rtol=1e-12, atol=1e-12)
    d = oracle_mod.Oracle(water648, seed=3, lj_long_mode=2, **p)
    assert d.jump_respa1(20, 1.0, 2, 3) == 0
    assert d.counters()[2] == 0 and d.counters()[0] > 0
    T = 0.5 * (water648.mass[:, None] * d.state()[1] ** 2).sum() / 418.4 * 2 / (3 * w.n * 0.0019872041)
    assert 200 < T < 1200


def test_bjaoajb_is_baoab_without_jumps_and_keeps_temperature(oracle_mod, water648):
    """BJAOAJB with empty jump ranges is BAOAB on F0 = full force bit for bit;
    with jumps it keeps the temperature of the water box near 300 K."""
    p = dict(r_cut=9.0, r_split=9.6, h_switch=0.5, skin=0.2, skin_outer=0.3)
    a = oracle_mod.Oracle(water648, seed=4, **p)
    b = oracle_mod.Oracle(water648, seed=4, **p)
    a.bjaoajb(20)
    b.baoab(20)
    xa, va, _, _ = a.state()
    xb, vb, _, _ = b.state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    c = oracle_mod.Oracle(water648, seed=4, r_cut=9.0, r_split=5.0, h_switch=0.5, skin=0.2, skin_outer=0.3)
    assert c.bjaoajb(60) == 0
    assert c.counters()[1] > 0
    v = c.state()[1]
    T = (water648.mass[:, None] * v * v).sum() / 418.4 / (3 * water648.n * 0.0019872042586)
    assert 240 < T < 360, T


def test_lists_cover_the_current_shells_during_dynamics(oracle_mod, water648):
    """Verlet validity of the rebuild rule (reading 11): after 300 JUMP steps
    behind a thin 0.2 A skin (the rule fires many times; the outer candidates
    have a wide skin, so their own rule does not mask it), every non-excluded
    pair whose current distance lies in a ring's range is in that ring's
    list, every O-O pair in the LJ range is in the LJ list, and every list
    entry is still within twice the skin of its shell."""
    skin = 0.2
    o = oracle_mod.Oracle(water648, r_cut=9.0, r_split=5.0, h_switch=0.5, r_mid=5.5, dsf_alpha=0.2,
                          skin=skin, skin_outer=1.0, seed=5)
    o.jump(300)
    assert o.errors == 0
    assert o.counters()[5] >= 5                               # list rebuilds (the outer rule, at 0.4 A, fires less)
    x = o.state()[0]
    L = water648.box
    n = water648.n
    mol = np.arange(n) // 3
    is_o = water648.type == 0
    for i in np.random.default_rng(2).choice(n, 40, replace=False):
        d = x[i] - x
        d -= L * np.round(d / L)
        r = np.sqrt((d * d).sum(1))
        ok = (np.arange(n) != i) & (mol != mol[i])
        for kind, lo, hi, extra in ((0, 4.5, 5.5, ok), (1, 5.5, 9.0, ok), (4, 4.5, 9.0, ok & is_o & is_o[i])):
            have = o.list_of(kind, i)
            need = np.flatnonzero(extra & (r >= lo) & (r < hi))
            assert np.isin(need, have).all(), (i, kind)
            assert ((r[have] >= lo - 2 * skin) & (r[have] < hi + 2 * skin)).all(), (i, kind)
