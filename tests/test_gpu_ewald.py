"""Parity of the CUDA path with the oracle under Ewald electrostatics
(coulomb_mode 1): real-space pairs erfc(a r)/r split by chi (Sec. 3.1), the
smooth-PME reciprocal part, the self and exclusion terms, and the integrators
that place the reciprocal part in F0 (JUMP, BJAOAJB) or at the outer level
(JUMP-RESPA, JUMP-RESPA1, Sec. 2.3).

Bars as in the DSF parity tests: per-atom gradient error <= 1e-12 (FP64) and
<= 1e-5 (mixed); identical accepted-jump events and positions within 1e-6 A
over 100 steps in FP64 mode.
"""
import numpy as np
import pytest

from test_gpu_parity import force_err, pos_err, sorted_events

pytestmark = pytest.mark.gpu

EWALD = dict(r_cut=9.0, r_split=5.0, h_switch=0.5, r_mid=5.5, dsf_alpha=0.35, gamma=1.0,
             temperature=300.0, eps0=0.1, eps_mode=1, skin=0.2, skin_outer=0.3,
             coulomb_mode=1, pme_order=6, pme_spacing=0.8)


@pytest.fixture(scope="module")
def M():
    import paper_2412_15073_gb300 as M
    M.load_library()
    return M


def make(M, oracle_mod, sys, precision, seed=0, graphs=True, **kw):
    p = dict(EWALD)
    p.update(kw)
    e = M.Engine(precision=precision, seed=seed, event_log_cap=1 << 21, graphs=graphs)
    e.set_system(0, sys, **p)
    o = oracle_mod.Oracle(sys, seed=seed, replica=0, **p)
    return e, o


def perturbed(w, seed=3):
    w = w.copy()
    w.x = (w.x + np.random.default_rng(seed).normal(scale=0.05, size=w.x.shape)) % w.box
    return w


# spacing 0.8 A gives K = 24 on the 18.6 A box, 0.7 A an odd K = 27, 1.6 A
# K = 12, where the 13-point region of a grid brick wraps onto itself
@pytest.mark.parametrize("spacing,order", [(0.8, 6), (0.7, 4), (0.8, 8), (1.6, 6)])
@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-5)])
def test_ewald_gradients(M, oracle_mod, water648, precision, tol, spacing, order):
    w = perturbed(water648)
    e, o = make(M, oracle_mod, w, precision, pme_spacing=spacing, pme_order=order)
    total, _ = o.gradient(0)
    errs = {}
    for mode in range(7):
        g = e.gradient(mode)
        ref, _ = o.gradient(mode)
        # partial sums against the total force: the chi-split parts, the
        # reciprocal part, and the nonbonded sum, which under Ewald is the
        # difference of a real-space and a reciprocal part each larger than it
        errs[mode] = force_err(g, ref, total if mode in (2, 3, 4, 6) else None)
    print("Ewald per-atom relative gradient error by mode:", errs)
    assert max(errs.values()) <= tol, errs
    # the reciprocal part is a real force here, not a rounding residue
    g6, _ = o.gradient(6)
    assert np.sqrt((g6 ** 2).sum(1).mean()) > 1.0


@pytest.mark.parametrize("precision,rtol", [(0, 1e-12), (1, 1e-6)])
def test_ewald_energy(M, oracle_mod, water648, precision, rtol):
    w = perturbed(water648)
    e, o = make(M, oracle_mod, w, precision)
    ob = e.observables()
    ref = o.energy()
    # pe_coul = real space + reciprocal + self + exclusion terms: a sum of terms
    # of size ~2e4 kcal/mol (the self term), so the bar is relative to that scale
    scale = abs(ob["pe_coul"]) + 2e4
    assert abs(ob["pe_coul"] - ref[3]) <= rtol * scale, (ob["pe_coul"], ref[3])
    assert ob["pe_lj"] == pytest.approx(ref[2], rel=max(rtol, 1e-11))


def test_ewald_jump_trajectory_and_events_fp64(M, oracle_mod, water648):
    e, o = make(M, oracle_mod, water648, 0, seed=7, ring_r=[6.0, 7.5])
    o.events_enable(1 << 22)
    e.jump(100)
    o.jump(100)
    xg, vg, _, _ = e.state()
    xo, vo, _, _ = o.state()
    ev_g, ev_o = sorted_events(e.events()), sorted_events(o.events())
    assert len(ev_o) > 100
    assert np.array_equal(ev_g, ev_o), (len(ev_g), len(ev_o))
    assert pos_err(xg, xo, water648.box) < 1e-6
    assert np.abs(vg - vo).max() < 1e-4


@pytest.mark.parametrize("integ,args", [("jump_respa1", (25, 1.0, 2, 2)), ("jump_respa", (50, 1.0, 2)),
                                        ("baoab_respa1", (25, 1.0, 2, 2)), ("bjaoajb", (100, 1.0))])
def test_ewald_multistep_trajectories_fp64(M, oracle_mod, water648, integ, args):
    """the reciprocal part at the outer level (RESPA kinds) or in F0 (BJAOAJB)"""
    e, o = make(M, oracle_mod, water648, 0, seed=11)
    o.events_enable(1 << 22)
    getattr(e, integ)(*args)
    getattr(o, integ)(*args)
    xg, vg, _, _ = e.state()
    xo, vo, _, _ = o.state()
    assert np.array_equal(sorted_events(e.events()), sorted_events(o.events()))
    assert pos_err(xg, xo, water648.box) < 1e-6
    assert np.abs(vg - vo).max() < 1e-4
    assert e.observables()["step"] == o.step


@pytest.mark.parametrize("integ,args", [("jump_respa1", (40, 1.0, 2, 3)), ("jump", (64, 1.0))])
def test_ewald_graphs_replay_plain_launches(M, oracle_mod, water648, integ, args):
    """mixed mode: CUDA-graph chunks (cuFFT inside the capture) equal plain launches bit for bit"""
    out = []
    for graphs in (True, False):
        e, _ = make(M, oracle_mod, water648, 1, seed=13, graphs=graphs)
        getattr(e, integ)(*args)
        x, v, _, _ = e.state()
        out.append((x, v, e.observables()["jump_accepts"]))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]


def test_ewald_and_dsf_replicas_side_by_side(M, oracle_mod, water648):
    """replicas of one context with different electrostatics and grids: each
    matches its own oracle (grid offsets, per-replica plans); odd B-spline
    orders are refused"""
    w1 = perturbed(water648, seed=5)
    cfgs = [dict(EWALD, coulomb_mode=0, dsf_alpha=0.2), dict(EWALD), dict(EWALD, pme_spacing=0.7, pme_order=4)]
    syss = [water648, w1, perturbed(water648, seed=9)]
    e = M.Engine(precision=0, seed=3, max_replicas=3)
    for r, (s, p) in enumerate(zip(syss, cfgs)):
        e.set_system(r, s, **p)
    with pytest.raises(M.MDError):
        e.set_system(2, syss[2], **dict(EWALD, pme_order=5))
    for r, (s, p) in enumerate(zip(syss, cfgs)):
        o = oracle_mod.Oracle(s, seed=3, replica=r, **p)
        total, _ = o.gradient(0)
        for mode in (0, 5, 6):
            ref, _ = o.gradient(mode)
            assert force_err(e.gradient(mode, replica=r), ref, total if mode == 6 else None) <= 1e-12, (r, mode)
        assert abs(e.observables(r)["pe_coul"] - o.energy()[3]) <= 1e-12 * 3e4


@pytest.mark.parametrize("precision", [0, 1])
def test_ewald_nve_energy_error_is_second_order(M, oracle_mod, water648, precision):
    """Velocity Verlet (BAOAB at gamma = 0) on the full Ewald force from a
    strained start (the system heats from 300 K to about 1100 K): the total
    energy pe + ke of the path's own energy routine fluctuates by O(dt^2), so
    halving dt divides its largest excursion by about 4. Forces that were not
    the gradient of that energy (a reciprocal force off by a factor, a missing
    exclusion correction) leave an error that does not shrink with dt."""
    w = perturbed(water648, seed=21)
    drift = {}
    for dt, n in ((0.25, 25), (0.125, 50)):
        e, _ = make(M, oracle_mod, w, precision, gamma=0.0)
        es = []
        for _ in range(16):
            ob = e.observables()
            es.append(ob["ke"] + ob["pe_bond"] + ob["pe_angle"] + ob["pe_lj"] + ob["pe_coul"])
            e.baoab(n, dt_fs=dt)
        drift[dt] = np.abs(np.array(es) - es[0]).max()
    print("NVE largest total-energy excursion (kcal/mol) by dt:", drift)
    assert 3.2 < drift[0.25] / drift[0.125] < 4.8, drift
    assert drift[0.125] < 1e-3 * abs(es[0]) + 3.0, drift


def test_ewald_weak_force_regime(M, oracle_mod, water648):
    """the paper's 96,000-atom setting (a = 0.42/A, short cutoff 6 A, eps0 =
    0.01): jumped forces of 1e-6 kcal/mol/A at the outer ring, acceptance
    ratios within 1e-8 of 1. FP64: events identical to the oracle and no bound
    flag; mixed: no bound flag either, though its FP32 ratios round above 1"""
    kw = dict(dsf_alpha=0.42, r_split=6.0, ring_r=[6.25, 7.0, 8.5], eps0=0.01)
    e, o = make(M, oracle_mod, water648, 0, seed=17, **kw)
    o.events_enable(1 << 23)
    e.jump(10)
    o.jump(10)
    assert o.errors == 0 and e.observables()["error_flags"] == 0
    assert np.array_equal(sorted_events(e.events()), sorted_events(o.events()))
    assert pos_err(e.state()[0], o.state()[0], water648.box) < 1e-6
    em, _ = make(M, oracle_mod, water648, 1, seed=17, **kw)
    em.jump_respa1(40, 1.0, 2, 3)
    ob = em.observables()
    assert ob["error_flags"] == 0 and ob["jump_proposals"] > 0


def test_ewald_batched_replicas_equal_solo_runs_mixed(M, oracle_mod, water648):
    """mixed precision: replicas with their own grids (24^3 and 27^3, orders 6
    and 4) advanced in one context give the same bits as each run alone (exact
    fixed-point charge sums, one transform per replica)"""
    w2 = perturbed(water648, seed=8)
    cfgs = [(water648, dict(EWALD)), (w2, dict(EWALD, pme_spacing=0.7, pme_order=4))]
    e = M.Engine(precision=1, seed=21, max_replicas=2)
    for r, (s, p) in enumerate(cfgs):
        e.set_system(r, s, **p)
    e.jump_respa1(12, 1.0, 2, 3)
    for r, (s, p) in enumerate(cfgs):
        solo = M.Engine(precision=1, seed=21, max_replicas=2)
        # the replica index keys its random streams: run it in the same slot
        if r == 1:
            solo.set_system(0, s, **p)
        solo.set_system(r, s, **p)
        solo.jump_respa1(12, 1.0, 2, 3)
        xb, vb, _, _ = e.state(r)
        xs, vs, _, _ = solo.state(r)
        assert np.array_equal(xb, xs) and np.array_equal(vb, vs), r


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-5)])
def test_ewald_water_with_charged_beads(M, oracle_mod, precision, tol):
    """The heterogeneous system (water around a dense sphere of charged LJ
    beads, three LJ types) under Ewald with the headline's settings, scaled
    down to 6,000 atoms: gradients of modes 0, 3, 5 and 6 against the oracle,
    then 200 BAOAB steps at 1 fs (gamma 1/ps) that run with no error flag and
    keep the temperature in a sane range."""
    import bench
    from paper_2412_15073_gb300 import systems
    w = systems.water_with_beads(n_total=6000, n_beads=600, seed=2)
    p = dict(bench.EW_BAOAB, lj_long_mode=2, skin=0.5)
    e = M.Engine(precision=precision, seed=3)
    e.set_system(0, w, **(p | {"gamma": 50.0}))
    e.baoab(400, 0.5)                   # relaxation from the lattice start at strong friction
    x, v, _, _ = e.state()
    w.x, w.v = x, v
    e.close()
    e = M.Engine(precision=precision, seed=4)
    e.set_system(0, w, **p)
    o = oracle_mod.Oracle(w, seed=4, replica=0, **p)
    total, _ = o.gradient(0)
    # the ionic order of the bead sphere makes the net force on a bead a small
    # difference of a real-space and a reciprocal part much larger than it:
    # the error is measured against the larger of the net force and the
    # reciprocal part (the floor 0.01 F_rms as elsewhere)
    recip = o.ewald_recip_pme()[0]
    scale = np.maximum(np.linalg.norm(total, axis=1), np.linalg.norm(recip, axis=1))
    floor = 0.01 * np.sqrt((total * total).sum(1).mean())
    errs = {}
    for mode in (0, 3, 5, 6):
        d = np.linalg.norm(e.gradient(mode) - o.gradient(mode)[0], axis=1)
        errs[mode] = float((d / np.maximum(scale, floor)).max())
    print("water + beads, Ewald: per-atom gradient error by mode", errs)
    assert max(errs.values()) <= tol, errs
    e.baoab(200)
    ob = e.observables()
    assert ob["error_flags"] == 0 and 250 < ob["temperature"] < 400, ob
