"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars: per-atom gradient error <= 1e-12 (FP64 mode) and <= 1e-5 (mixed mode),
measured as |dF_i| / max(|F_i|, 0.01 F_rms); identical jump lists; identical
accepted-jump events and positions within 1e-6 A over 100 steps (FP64 mode);
sampled per-atom C' phases at 24,000 atoms.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

PARAMS = dict(r_cut=9.0, r_split=5.0, h_switch=0.5, r_mid=5.5, dsf_alpha=0.2, gamma=1.0,
              temperature=300.0, eps0=0.1, eps_mode=1, skin=0.2, skin_outer=0.3)


@pytest.fixture(scope="module")
def M():
    import paper_2412_15073_gb300 as M
    M.load_library()
    return M


def make(M, oracle_mod, sys, precision, seed=0, tpa=0, **kw):
    p = dict(PARAMS)
    p.update(kw)
    e = M.Engine(precision=precision, seed=seed, event_log_cap=1 << 21, threads_per_atom=tpa)
    e.set_system(0, sys, **p)
    o = oracle_mod.Oracle(sys, seed=seed, replica=0, **p)
    return e, o


def force_err(g, ref, scale=None):
    """max_i |dF_i| / max(|F_i|, 0.01 F_rms), F the force that moves the atom
    (scale, when given, is that force: the total for a partial sum)"""
    s = ref if scale is None else scale
    rms = np.sqrt((s * s).sum(1).mean())
    den = np.maximum(np.linalg.norm(s, axis=1), 0.01 * rms)
    return (np.linalg.norm(g - ref, axis=1) / den).max()


def pos_err(xa, xb, L):
    d = xa - xb
    d -= L * np.round(d / L)
    return np.abs(d).max()


def sorted_events(ev):
    ev = np.asarray(ev, dtype=np.int64).reshape(-1, 6)
    return ev[np.lexsort(ev.T[::-1])]


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-5)])
def test_gradients(M, oracle_mod, water648, precision, tol):
    w = water648.copy()
    w.x = (w.x + np.random.default_rng(3).normal(scale=0.05, size=w.x.shape)) % w.box
    e, o = make(M, oracle_mod, w, precision)
    total, _ = o.gradient(0)
    errs, own = {}, {}
    for mode in range(6):
        g = e.gradient(mode)
        ref, _ = o.gradient(mode)
        own[mode] = force_err(g, ref)
        # the chi-split parts (3 short, 4 long) are measured against the total
        # force acting on the atom; the others are forces in their own right
        errs[mode] = force_err(g, ref, total if mode in (3, 4) else None)
    print("per-atom relative gradient error by mode:", errs, "own-scale:", own)
    assert max(errs.values()) <= tol, errs


def test_fixed_point_forces_do_not_depend_on_threads_per_atom(M, oracle_mod, water648, monkeypatch):
    """Mixed mode: the pair gradients are the same bits for every number of
    threads per atom, and for the half-list kernels (each unique pair once,
    both atoms served by integer atomics) as for the full-list ones: gradient
    modes 0, 2, 3, 4 and 5, and with the LJ long part deterministic at the slow
    level (lj_long_mode 2, where mode 3 may run half and mode 5 may not)."""
    gs = []
    for tpa in (1, 2, 4, 8):
        e, _ = make(M, oracle_mod, water648, 1, tpa=tpa)
        gs.append(np.stack([e.gradient(m) for m in (0, 2, 3, 4, 5)]))
    for var in (17, 18, 20, 24):
        monkeypatch.setenv("MDJ_FORCE_VARIANT", str(var))
        e, _ = make(M, oracle_mod, water648, 1)
        gs.append(np.stack([e.gradient(m) for m in (0, 2, 3, 4, 5)]))
        e.close()
    for k, g in enumerate(gs[1:]):
        assert np.array_equal(g, gs[0]), k
    ref2 = None
    for var in (2, 20):
        monkeypatch.setenv("MDJ_FORCE_VARIANT", str(var))
        e, _ = make(M, oracle_mod, water648, 1, lj_long_mode=2)
        g = np.stack([e.gradient(m) for m in (0, 3, 4, 5, 6)])
        e.close()
        if ref2 is None:
            ref2 = g
        else:
            assert np.array_equal(g, ref2)


def test_cluster_tiles_give_the_per_atom_bits():
    """The cluster-tile kernels (variant 33, opt-in through MDJ_TILES) need half
    the box to exceed the list radius plus a cluster's extent, so 648 atoms
    would fall back to the per-atom kernels; 6,591 atoms in a 40.3 A box (DSF,
    and Ewald real space with the LJ long part at the slow level) run them: the
    full, short, long and F0 gradients are the same bits as the
    thread-per-atom and half-list kernels'."""
    import paper_2412_15073_gb300 as M
    from paper_2412_15073_gb300 import systems
    import os
    w = systems.water_box(2197, box=40.3, seed=2)
    cases = [(dict(PARAMS), (0, 2, 3, 4, 5)),
             (dict(PARAMS, dsf_alpha=0.35, coulomb_mode=1, pme_order=6, pme_spacing=0.8, r_split=6.0,
                   lj_long_mode=2), (2, 3, 4))]
    old = os.environ.get("MDJ_FORCE_VARIANT")
    os.environ["MDJ_TILES"] = "1"           # the tiles are opt-in
    try:
        for p, modes in cases:
            ref = None
            for var in (1, 17, 33):
                os.environ["MDJ_FORCE_VARIANT"] = str(var)
                e = M.Engine(precision=1, seed=0)
                e.set_system(0, w, **p)
                g = np.stack([e.gradient(m) for m in modes])
                e.close()
                if ref is None:
                    ref = g
                else:
                    assert np.array_equal(g, ref), (var, p.get("coulomb_mode", 0))
    finally:
        os.environ.pop("MDJ_TILES", None)
        if old is None:
            os.environ.pop("MDJ_FORCE_VARIANT", None)
        else:
            os.environ["MDJ_FORCE_VARIANT"] = old


RINGS = [None, [], [4.8, 6.0, 7.5]]     # rings of r_mid (two), one ring, four rings


@pytest.mark.parametrize("ring_r", RINGS)
@pytest.mark.parametrize("precision", [0, 1])
def test_jump_lists_identical(M, oracle_mod, water648, precision, ring_r):
    e, o = make(M, oracle_mod, water648, precision, ring_r=ring_r)
    nonempty = np.zeros(5, dtype=int)
    for i in range(0, water648.n, 7):
        for kind in range(5):       # rings 0..3, LJ
            lg = e.get_list(kind, i)
            np.testing.assert_array_equal(lg, o.list_of(kind, i))
            nonempty[kind] += len(lg) > 0
    n_rings = 2 if ring_r is None else len(ring_r) + 1
    assert (nonempty[:n_rings] > 0).all() and (nonempty[n_rings:4] == 0).all() and nonempty[4] > 0


def test_baoab_trajectory_fp64(M, oracle_mod, water648):
    e, o = make(M, oracle_mod, water648, 0, seed=5)
    e.baoab(100)
    o.baoab(100)
    xg, vg, ig, _ = e.state()
    xo, vo, io, _ = o.state()
    assert pos_err(xg, xo, water648.box) < 1e-6
    assert np.abs(vg - vo).max() < 1e-5
    assert np.array_equal(ig, io)
    assert e.observables()["list_rebuilds"] == o.counters()[5]


@pytest.mark.parametrize("ring_r", RINGS)
def test_jump_trajectory_and_events_fp64(M, oracle_mod, water648, ring_r):
    e, o = make(M, oracle_mod, water648, 0, seed=7, ring_r=ring_r)
    o.events_enable(1 << 22)
    e.jump(100)
    o.jump(100)
    xg, vg, _, _ = e.state()
    xo, vo, _, _ = o.state()
    ev_g, ev_o = sorted_events(e.events()), sorted_events(o.events())
    assert len(ev_o) > 1000
    assert np.array_equal(ev_g, ev_o), (len(ev_g), len(ev_o))
    c = o.counters()
    ob = e.observables()
    assert (ob["jump_proposals"], ob["jump_accepts"], ob["bps_proposals"], ob["bps_accepts"]) == tuple(c[:4])
    assert pos_err(xg, xo, water648.box) < 1e-6
    assert np.abs(vg - vo).max() < 1e-5
    assert ob["error_flags"] == 0 and o.errors == 0


@pytest.mark.parametrize("how", ["baoab_respa", "baoab_respa1", "jump_respa", "jump_respa1"])
def test_multiple_time_step_family_fp64(M, oracle_mod, water648, how):
    e, o = make(M, oracle_mod, water648, 0, seed=11)
    args = {"baoab_respa": (25, 1.0, 2), "jump_respa": (25, 1.0, 2),
            "baoab_respa1": (10, 1.0, 2, 3), "jump_respa1": (10, 1.0, 2, 3)}[how]
    getattr(e, how)(*args)
    getattr(o, how)(*args)
    xg, vg, _, _ = e.state()
    xo, vo, _, _ = o.state()
    assert e.observables()["step"] == o.step
    assert pos_err(xg, xo, water648.box) < 1e-6, how
    assert np.abs(vg - vo).max() < 1e-5, how


@pytest.mark.parametrize("precision", [0, 1])
def test_fused_inner_steps_equal_separate_launches(M, oracle_mod, water648, monkeypatch, precision):
    """The inner steps of the multiple-time-step drivers run fused (one launch
    for all inner steps of a cycle, blocks of whole molecules): the same bits
    as the separate kick, A-O-A and bonded launches, for the four drivers."""
    runs = {"baoab_respa": (12, 1.0, 2), "baoab_respa1": (5, 1.0, 2, 3), "jump_respa": (12, 1.0, 3),
            "jump_respa1": (5, 1.0, 2, 2)}
    for how, args in runs.items():
        got = []
        for fused in (True, False):
            if fused:
                monkeypatch.setenv("MDJ_FUSED_INNER", "1")
            else:
                monkeypatch.delenv("MDJ_FUSED_INNER", raising=False)
            e, _ = make(M, oracle_mod, water648, precision, seed=14)
            getattr(e, how)(*args)
            x, v, img, xb = e.state()
            ob = e.observables()
            got.append((x, v, img, xb, ob["list_rebuilds"], ob["step"]))
            e.close()
        a, b = got
        for k in range(4):
            assert np.array_equal(a[k], b[k]), (how, k)
        assert a[4:] == b[4:], how


def test_jump_mixed_precision_tracks_oracle(M, oracle_mod, water648):
    """Mixed mode: FP32 pair math and jump loops against the FP64 oracle. Over
    10 steps the accepted jumps agree except near rare ties (a flip changes
    one atom's velocity, after which that atom's later events differ), and the
    positions stay within 1e-3 A."""
    e, o = make(M, oracle_mod, water648, 1, seed=7)
    o.events_enable(1 << 22)
    e.jump(10)
    o.jump(10)
    ev_g = {tuple(r) for r in e.events().tolist()}
    ev_o = {tuple(r) for r in o.events().tolist()}
    flips = len(ev_g ^ ev_o)
    print("mixed-mode events:", len(ev_o), "differing:", flips)
    assert flips <= 0.02 * len(ev_o), (flips, len(ev_o))
    xg = e.state()[0]
    xo = o.state()[0]
    d = xg - xo
    d -= water648.box * np.round(d / water648.box)
    err = np.sqrt((d * d).sum(1))
    print("mixed-mode position error after 10 steps: mean", err.mean(), "max", err.max())
    assert err.mean() < 1e-3


@pytest.mark.parametrize("ring_r", [None, [4.8, 6.0, 7.5]])
def test_jump_mixed_precision_statistics(M, oracle_mod, water648, ring_r):
    """Over 200 steps the mixed-mode path keeps the oracle's jump statistics:
    proposals per atom-step and accepted fractions agree within 3 %."""
    e, o = make(M, oracle_mod, water648, 1, seed=8, ring_r=ring_r)
    e.jump(200)
    o.jump(200)
    ob = e.observables()
    c = o.counters()
    for got, ref in ((ob["jump_proposals"], c[0]), (ob["jump_accepts"], c[1])):
        assert abs(got / ref - 1) < 0.03, (got, ref)
    assert abs(ob["bps_proposals"] / max(c[2], 1) - 1) < 0.25
    assert ob["error_flags"] == 0


@pytest.mark.parametrize("ring_r", [None, [5.0, 5.5, 7.0]])
def test_sampled_cprime_phase_at_24000_atoms(M, oracle_mod, ring_r):
    """One C' phase on 24,000 atoms (8,000 waters, 62.1 A) on the GPU in both
    precisions, checked atom by atom against the oracle on 300 sampled atoms."""
    from paper_2412_15073_gb300 import systems
    w = systems.water_box(8000, box=62.1, seed=0)
    p = dict(PARAMS, skin=0.5, skin_outer=1.5, ring_r=ring_r)
    o = oracle_mod.Oracle(w, seed=3, replica=0, **p)
    rng = np.random.default_rng(1)
    idx = rng.choice(w.n, 300, replace=False)
    mt = w.mass / 418.4
    tau2 = 0.0005
    for precision, rtol, frac in ((0, 1e-10, 1.0), (1, 2e-5, 0.98)):
        e = M.Engine(precision=precision, seed=3)
        e.set_system(0, w, **p)
        e.run_phase(0, tau2, s0=123, half=0, accel_mode=M.GRAD_F0)
        vg = e.state()[1]
        good = 0
        for i in idx:
            a = -o.gradient_atom(oracle_mod.GRAD_F0, i) / mt[i]
            vo, _, _ = o.cprime_one(i, w.v[i], a, tau2, 123, 0)
            good += np.abs(vg[i] - vo).max() <= rtol * max(np.abs(vo).max(), 1.0)
        assert good >= frac * len(idx), (precision, good)
        e.close()


def test_batched_replicas(M, oracle_mod):
    """Three replicas of uneven size in one launch per step: each matches the
    oracle run with its own Philox key (FP64), and replica 0 of a mixed batch
    equals a mixed solo run bit for bit."""
    from paper_2412_15073_gb300 import systems
    sizes = [216, 290, 250]
    syss = [systems.water_box(n, seed=10 + k) for k, n in enumerate(sizes)]
    p = dict(PARAMS)
    e = M.Engine(precision=0, seed=9, max_replicas=3)
    for r, s in enumerate(syss):
        e.set_system(r, s, **p)
    e.jump(40)
    for r, s in enumerate(syss):
        o = oracle_mod.Oracle(s, seed=9, replica=r, **p)
        o.jump(40)
        e.n[r] = s.n
        assert pos_err(e.state(r)[0], o.state()[0], s.box) < 1e-6, r
    eb = M.Engine(precision=1, seed=9, max_replicas=3)
    for r, s in enumerate(syss):
        eb.set_system(r, s, **p)
    es = M.Engine(precision=1, seed=9)
    es.set_system(0, syss[0], **p)
    eb.jump(40)
    es.jump(40)
    xb, vb, _, _ = eb.state(0)
    xs, vs, _, _ = es.state(0)
    assert np.array_equal(xb, xs) and np.array_equal(vb, vs)


def test_resume_bit_exact_on_gpu(M, oracle_mod, water648):
    a, _ = make(M, oracle_mod, water648, 1, seed=6)
    a.jump(40)
    xa, va, _, _ = a.state()
    b, _ = make(M, oracle_mod, water648, 1, seed=6)
    b.jump(20)
    x, v, img, xb, xo = b.state(outer=True)
    c, _ = make(M, oracle_mod, water648, 1, seed=6)
    c.set_state(0, x, v, img, xb, xo, step=20)
    c.jump(20)
    xc, vc, _, _ = c.state()
    assert np.array_equal(xa, xc) and np.array_equal(va, vc)


def test_energy_observables(M, oracle_mod, water648):
    e, o = make(M, oracle_mod, water648, 0, seed=2)
    e.jump(10)
    o.jump(10)
    ob = e.observables()
    ref = o.energy()
    got = np.array([ob["pe_bond"], ob["pe_angle"], ob["pe_lj"], ob["pe_coul"]])
    np.testing.assert_allclose(got, ref, rtol=1e-9, atol=1e-9)
    v = o.state()[1]
    ke = 0.5 * (water648.mass[:, None] * v * v).sum() / 418.4
    assert ob["ke"] == pytest.approx(ke, rel=1e-9)


def test_jump_is_baoab_without_jump_range_on_gpu(M, oracle_mod, water648):
    p = dict(r_split=9.6)
    a, _ = make(M, oracle_mod, water648, 1, seed=4, **p)
    b, _ = make(M, oracle_mod, water648, 1, seed=4, **p)
    a.jump(30)
    b.baoab(30)
    xa, va, _, _ = a.state()
    xb, vb, _, _ = b.state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)


def test_invalid_inputs_are_rejected(M, water648):
    e = M.Engine(precision=1)
    with pytest.raises(M.MDError) as ex:
        e.set_system(0, water648, r_cut=9.0, skin=0.5, skin_outer=1.0)   # box < 2 (r_cut + skin_outer)
    assert ex.value.code == -1
    with pytest.raises(M.MDError):
        e.jump(1)                                                         # no system yet
    with pytest.raises(M.MDError):
        e.set_system(1, water648)                                         # replica out of range
    for bad in ([6.0, 5.5], [4.0], [9.5], [5.0, 5.5, 6.0, 7.0]):
        with pytest.raises((M.MDError, ValueError)):
            e.set_system(0, water648, ring_r=bad)                        # ring edges not inside (r_c-h, r_E)


def test_uncharged_lj_fluid_and_degenerate_calls(M, oracle_mod):
    """Degenerate cases. An uncharged Lennard-Jones lattice (512 argon-like
    atoms, 30.4 A): the Coulomb rings are empty, so JUMP is BAOAB with the LJ
    bounces (J') only, and the FP64 bounces and positions equal the oracle's
    over 100 steps of 2 fs. Zero steps leave the state alone; an empty system
    is refused."""
    from paper_2412_15073_gb300 import systems
    n, a = 8, 3.8
    g = np.stack(np.meshgrid(*(np.arange(n),) * 3, indexing="ij"), -1).reshape(-1, 3) * a + 0.5
    w = systems.point_charges(g, n * a, 0.0, 39.948, seed=3, temperature=120.0, lj_eps=0.238, lj_sigma=3.4)
    p = dict(PARAMS, temperature=120.0, skin=0.3, skin_outer=0.6)
    e = M.Engine(precision=0, seed=4, event_log_cap=1 << 20)
    e.set_system(0, w, **p)
    o = oracle_mod.Oracle(w, seed=4, replica=0, **p)
    o.events_enable(1 << 20)
    x0 = e.state()[0]
    e.jump(0, 2.0)
    assert np.array_equal(e.state()[0], x0) and e.observables()["step"] == 0
    e.jump(100, 2.0)
    o.jump(100, 2.0)
    ev_g, ev_o = sorted_events(e.events()), sorted_events(o.events())
    assert len(ev_o) > 50 and np.array_equal(ev_g, ev_o), (len(ev_g), len(ev_o))
    assert pos_err(e.state()[0], o.state()[0], w.box) < 1e-6
    ob = e.observables()
    assert ob["jump_proposals"] == 0 and ob["bps_accepts"] == len(ev_o) and ob["error_flags"] == 0
    e.close()
    empty = systems.point_charges(np.zeros((0, 3)), 30.0, 0.0, 1.0)
    with pytest.raises(M.MDError):
        M.Engine(precision=1).set_system(0, empty)


def test_failures_are_reported_as_status(M, water648):
    """Failure detection without a GPU fault, the failure made on the host:
    an event log smaller than the run's accepted jumps makes md_get_events
    return MD_EOVERFLOW (the kernels stop writing at its end), and a
    non-finite velocity handed to md_set_state is caught by the A O A
    update's check, so the step call returns MD_ENONFINITE. Every device
    loop is bounded (proposal and sampler caps), so neither case hangs."""
    e = M.Engine(precision=1, seed=2, event_log_cap=16)
    e.set_system(0, water648, **PARAMS)
    e.jump(5)
    with pytest.raises(M.MDError) as ex:
        e.events()
    assert ex.value.code == -3
    x, v, img, xb = e.state()
    v[7] = np.nan
    e.set_state(0, x, v, img, xb)
    with pytest.raises(M.MDError) as ex:
        e.jump(1)
    assert ex.value.code == -6
    e.close()


def test_velocity_phase_variants_are_identical(M, oracle_mod, water648, monkeypatch):
    """The launch variants the autotuner chooses between (four occupancy
    targets, with or without the rate ordering, one thread per atom or lanes
    fed from a queue of atoms) compute the same values bit for bit (mixed
    mode, 20 JUMP steps), on one system and on a batch of three replicas
    (where the queue kernel moves lanes between replicas)."""
    from paper_2412_15073_gb300 import systems
    ref = None
    for var in range(16):
        monkeypatch.setenv("MDJ_VPHASE_VARIANT", str(var))
        e, _ = make(M, oracle_mod, water648, 1, seed=12)
        e.jump(20)
        x, v, _, _ = e.state()
        ob = e.observables()
        got = (x, v, ob["jump_proposals"], ob["jump_accepts"], ob["bps_proposals"])
        if ref is None:
            ref = got
        else:
            assert np.array_equal(x, ref[0]) and np.array_equal(v, ref[1]) and got[2:] == ref[2:], var
        e.close()
    syss = [systems.water_box(n, seed=20 + k) for k, n in enumerate([216, 343, 250])]
    refb = None
    for var in (0, 4, 8, 9, 12):
        monkeypatch.setenv("MDJ_VPHASE_VARIANT", str(var))
        e = M.Engine(precision=1, seed=13, max_replicas=3)
        for r, s in enumerate(syss):
            e.set_system(r, s, **PARAMS)
        e.jump(15)
        got = [e.state(r)[1] for r in range(3)] + [e.observables(r)["jump_proposals"] for r in range(3)]
        if refb is None:
            refb = got
        else:
            for r in range(3):
                assert np.array_equal(got[r], refb[r]), (var, r)
            assert got[3:] == refb[3:], var
        e.close()


@pytest.mark.parametrize("how", ["jump", "jump_respa"])
def test_fused_cprime_pairs_equal_single_phases(M, oracle_mod, water648, how):
    """Mixed mode runs the adjacent C' phases of consecutive steps in one
    launch; that must give the same values bit for bit as one call per step
    (where every phase has a launch of its own)."""
    a, _ = make(M, oracle_mod, water648, 1, seed=13)
    b, _ = make(M, oracle_mod, water648, 1, seed=13)
    if how == "jump":
        a.jump(12)
        for _ in range(12):
            b.jump(1)
    else:
        a.jump_respa(6, 1.0, 2)
        for _ in range(6):
            b.jump_respa(1, 1.0, 2)
    xa, va, _, _ = a.state()
    xb, vb, _, _ = b.state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    oa, ob = a.observables(), b.observables()
    assert oa["jump_proposals"] == ob["jump_proposals"] and oa["jump_accepts"] == ob["jump_accepts"]


@pytest.mark.parametrize("how,args", [("jump", (40,)), ("baoab", (40,)), ("jump_respa", (20, 1.0, 2)),
                                      ("baoab_respa1", (12, 1.0, 2, 2)), ("jump_respa1", (12, 1.0, 2, 2))])
def test_graph_replays_equal_plain_launches(M, oracle_mod, water648, how, args):
    """Long calls replay CUDA graphs of 16-step chunks; the trajectory, the
    counters and the step count equal those of plain launches, and a second
    call reuses the graph and continues the same trajectory."""
    runs = []
    for graphs in (True, False):
        e = M.Engine(precision=1, seed=21, event_log_cap=0, graphs=graphs)
        e.set_system(0, water648, **PARAMS)
        getattr(e, how)(*args)
        getattr(e, how)(*args)
        x, v, img, _ = e.state()
        ob = e.observables()
        runs.append((x, v, img, ob))
        e.close()
    (xa, va, ia, oa), (xb, vb, ib, ob) = runs
    assert np.array_equal(xa, xb) and np.array_equal(va, vb) and np.array_equal(ia, ib)
    for k in ("step", "jump_proposals", "jump_accepts", "bps_proposals", "list_rebuilds"):
        assert oa[k] == ob[k], k


def test_batched_ensemble_of_64_replicas(M, oracle_mod):
    """The batched ensemble: 64 replicas of 216-2000 waters (sizes from seed
    1), each in its own box, advanced together in FP64; four sampled replicas
    (the smallest, the largest and two others) follow their own oracle runs
    to 1e-6 A over 10 JUMP steps."""
    from paper_2412_15073_gb300 import systems
    sizes = systems.replica_sizes(64, seed=1)
    syss = [systems.water_box(n, seed=100 + k) for k, n in enumerate(sizes)]
    e = M.Engine(precision=0, seed=3, max_replicas=64)
    for r, s in enumerate(syss):
        e.set_system(r, s, **PARAMS)
    e.jump(10)
    pick = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), 17, 40})
    for r in pick:
        o = oracle_mod.Oracle(syss[r], seed=3, replica=r, **PARAMS)
        o.jump(10)
        assert pos_err(e.state(r)[0], o.state()[0], syss[r].box) < 1e-6, r
        assert e.observables(r)["jump_accepts"] == o.counters()[1], r
    e.close()


def test_million_atom_heterogeneous_sampled(M, oracle_mod):
    """The 1,000,000-atom system (water around a dense sphere of 50,002
    charged LJ beads in rock-salt order, 229 A box) in mixed precision:
    gradients of 40 sampled atoms within 1e-5 of the oracle's, and one C'
    phase of 100 sampled atoms (oracle with per-atom lists, since its O(N^2)
    list build is out of reach). On a bead the net force is a small difference
    of pair forces about ten times larger (its six nearest neighbours carry the
    opposite charge), so the error is measured against the larger of the net
    force and one tenth of the sum of the pair-force magnitudes (the error of
    an FP32 sum scales with the magnitudes summed)."""
    from paper_2412_15073_gb300 import systems
    w = systems.water_with_beads()
    p = dict(PARAMS, r_cut=10.0, skin=0.5, skin_outer=1.5)
    e = M.Engine(precision=1, seed=5)
    e.set_system(0, w, **p)
    o = oracle_mod.Oracle(w, seed=5, replica=0, lazy_lists=True, **p)
    rng = np.random.default_rng(7)
    n_w = 3 * 316_666
    idx = np.concatenate([rng.choice(n_w, 30, replace=False), n_w + rng.choice(w.n - n_w, 10, replace=False)])
    def abs_sum(i, weight):
        """sum over the partners of atom i of |d/dr (weighted U)| (oracle pair terms)"""
        d = w.x - w.x[i]
        d -= w.box * np.round(d / w.box)
        r = np.sqrt((d * d).sum(1))
        mol = np.arange(w.n) // 3
        near = np.flatnonzero((r < p["r_cut"]) & (np.arange(w.n) != i) &
                              ~((mol == mol[i]) & (i < n_w) & (np.arange(w.n) < n_w)))
        return sum(abs(o.pair_dudr(int(w.type[i]), int(w.type[j]), w.charge[i] * w.charge[j], r[j], weight))
                   for j in near)

    for mode in (0, 3):
        g = e.gradient(mode)
        tot = e.gradient(0) if mode == 3 else g
        rms = np.sqrt((tot * tot).sum(1).mean())
        for i in idx:
            ref = o.gradient_atom(mode, int(i))
            den = max(np.linalg.norm(tot[i]), 0.01 * rms, 0.1 * abs_sum(int(i), 0 if mode == 0 else 1))
            assert np.linalg.norm(g[i] - ref) / den <= 1e-5, (mode, i)
    mt = w.mass / 418.4
    tau2 = 0.0005
    e.run_phase(0, tau2, s0=11, half=0, accel_mode=M.GRAD_F0)
    vg = e.state()[1]
    good = 0
    sample = rng.choice(w.n, 100, replace=False)
    for i in sample:
        a = -o.gradient_atom(oracle_mod.GRAD_F0, int(i)) / mt[i]
        vo, _, _ = o.cprime_one(int(i), w.v[i], a, tau2, 11, 0)
        good += np.abs(vg[i] - vo).max() <= 2e-5 * max(np.abs(vo).max(), 1.0)
    assert good >= 97, good
    e.close()


@pytest.mark.parametrize("workload", ["dsf_jump", "ewald_jump_respa1"])
def test_benchmark_workloads_sampled(M, oracle_mod, workload):
    """The benchmark workloads themselves (96,000-atom water, 98.6 A, with the
    benchmark's list settings): the DSF JUMP step (r_E 10 A, rings at 5.25 / 6
    / 7.5 A, 0.3 A skin) and the Ewald JUMP-RESPA1 cycle of the headline
    (a 0.42/A, PME order 6 on 125^3, r_c 6 A, one ring, LJ long part at the
    slow level). Gradients of 40 sampled atoms (F0 and full, or the short
    part and the slow level) within 1e-12 of the oracle's in FP64 and 1e-5 in
    mixed precision; one C' phase of 200 sampled atoms: in FP64 the accepted
    jumps are the oracle's and the velocities agree to 1e-10, in mixed
    precision at most one atom of the 200 ends differently (a decision flipped
    by FP32 rounding; about none are expected) and the count is printed.
    The oracle builds lists per atom (its O(N^2) build is out of reach here)."""
    import bench
    from paper_2412_15073_gb300 import systems
    w = systems.water_box(bench.N_MOL, box=bench.BOX, seed=0)
    ewald = workload == "ewald_jump_respa1"
    p = dict(bench.EW_JUMP if ewald else bench.DSF_JUMP)
    o = oracle_mod.Oracle(w, seed=6, replica=0, lazy_lists=True, **p)
    rng = np.random.default_rng(8)
    idx = rng.choice(w.n, 40, replace=False)
    phase_atoms = rng.choice(w.n, 200, replace=False)
    modes = (3, 6) if ewald else (0, 5)
    accel = M.GRAD_NB_SHORT if ewald else M.GRAD_F0
    tau2, s0, half = (0.001, 21, 0) if ewald else (0.0005, 17, 1)
    recip = None
    if ewald:
        # the slow level = the (1 - chi) LJ part (an oracle without Ewald gives it alone)
        # + the reciprocal part, computed once for all atoms
        o_lj = oracle_mod.Oracle(w, seed=6, replica=0, lazy_lists=True, **(p | {"coulomb_mode": 0}))
        recip = o.ewald_recip_pme()[0]

    def ref_grad(mode, i):
        if mode == 6:
            return o_lj.gradient_atom(6, int(i)) + recip[i]
        return o.gradient_atom(mode, int(i))

    refs = {mode: {int(i): ref_grad(mode, i) for i in idx} for mode in modes}
    o.events_enable(1 << 20)
    mt = w.mass / 418.4
    vo = {}
    for i in phase_atoms:
        a = -o.gradient_atom(int(accel), int(i)) / mt[i]
        vo[int(i)] = o.cprime_one(int(i), w.v[i], a, tau2, s0, half)[0]
    ev_o = {tuple(r) for r in o.events().tolist()}
    for precision, tol in ((0, 1e-12), (1, 1e-5)):
        e = M.Engine(precision=precision, seed=6, event_log_cap=1 << 22)
        e.set_system(0, w, **p)
        tot = e.gradient(0)
        rms = np.sqrt((tot * tot).sum(1).mean())
        for mode in modes:
            g = tot if mode == 0 else e.gradient(mode)
            for i in idx:
                den = max(np.linalg.norm(tot[i]), 0.01 * rms)
                err = np.linalg.norm(g[i] - refs[mode][int(i)]) / den
                assert err <= tol, (precision, mode, i, err)
        e.run_phase(0, tau2, s0=s0, half=half, accel_mode=accel)
        vg = e.state()[1]
        sel = set(int(i) for i in phase_atoms)
        ev_g = {tuple(r) for r in e.events().tolist() if r[3] in sel}
        differ = [int(i) for i in phase_atoms
                  if np.abs(vg[i] - vo[int(i)]).max() > (1e-10 if precision == 0 else 2e-5) * max(np.abs(vo[int(i)]).max(), 1.0)]
        print(f"{workload} precision {precision}: {len(ev_o)} oracle events on 200 atoms, "
              f"{len(ev_g ^ ev_o)} differing events, {len(differ)} atoms ending differently")
        if precision == 0:
            assert ev_g == ev_o
            assert not differ, differ
        else:
            assert len(differ) <= 1, differ
        assert e.observables()["error_flags"] == 0
        e.close()


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-5)])
def test_lj_long_mode_gradients(M, oracle_mod, water648, precision, tol):
    """The LJ long part deterministic: in F0 (mode 1, the paper's GPU
    variant) or at the slow level (mode 2): gradient modes against the
    oracle's, partial sums measured against the total force."""
    w = water648.copy()
    w.x = (w.x + np.random.default_rng(3).normal(scale=0.05, size=w.x.shape)) % w.box
    for lj_long_mode in (1, 2):
        e, o = make(M, oracle_mod, w, precision, lj_long_mode=lj_long_mode)
        total, _ = o.gradient(0)
        for mode in (0, 3, 4, 5, 6):
            ref, _ = o.gradient(mode)
            err = force_err(e.gradient(mode), ref, total if mode in (3, 4, 6) else None)
            assert err <= tol, (lj_long_mode, mode, err)


@pytest.mark.parametrize("how,kw", [("jump", dict(lj_long_mode=1)), ("bjaoajb", {}),
                                    ("bjaoajb", dict(lj_long_mode=1)), ("jump", dict(lj_long_mode=2)),
                                    ("jump_respa1", dict(lj_long_mode=2)), ("jump_respa", dict(lj_long_mode=2))])
def test_variant_trajectories_fp64(M, oracle_mod, water648, how, kw):
    """JUMP with the deterministic LJ long part, and the BJAOAJB splitting,
    follow the oracle in FP64: identical accepted-jump events and positions
    within 1e-6 A over 60 steps; no LJ bounces when the LJ long part is
    deterministic."""
    e, o = make(M, oracle_mod, water648, 0, seed=9, **kw)
    o.events_enable(1 << 22)
    args = {"jump_respa1": (10, 1.0, 2, 3), "jump_respa": (30, 1.0, 2)}.get(how, (60,))
    getattr(e, how)(*args)
    getattr(o, how)(*args)
    assert np.array_equal(sorted_events(e.events()), sorted_events(o.events()))
    assert pos_err(e.state()[0], o.state()[0], water648.box) < 1e-6
    ob = e.observables()
    assert ob["jump_accepts"] == o.counters()[1] > 0
    if kw.get("lj_long_mode"):
        assert ob["bps_proposals"] == 0


def test_bjaoajb_graphs_and_mixed(M, oracle_mod, water648):
    """Mixed-mode BJAOAJB: graph replays equal plain launches bit for bit."""
    runs = []
    for graphs in (True, False):
        e = M.Engine(precision=1, seed=23, graphs=graphs)
        e.set_system(0, water648, **PARAMS)
        e.bjaoajb(40)
        runs.append(e.state()[:2])
        e.close()
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])


@pytest.mark.parametrize("how", ["baoab", "jump"])
def test_plain_648_atom_workload_1000_steps_fp64(M, oracle_mod, how):
    """The plain workload as specified: 216 waters on the lattice from seed 0,
    DSF alpha 0.2 with a 9 A cutoff, split at 5 A, 1000 steps of 1 fs in FP64.
    The GPU run follows the oracle's to 1e-6 A for the first 100 steps; after
    that, rounding differences (summation order, fused multiply-adds) grow
    as in any chaotic system, so the last 900 steps are compared in law: the
    mean temperature over steps 200-1000 within 4 % and the jump counts within
    2 %."""
    from paper_2412_15073_gb300 import systems
    w = systems.water_box(216, box=18.643, seed=0)
    e = M.Engine(precision=0, seed=0)
    e.set_system(0, w, **PARAMS)
    o = oracle_mod.Oracle(w, seed=0, replica=0, **PARAMS)
    getattr(e, how)(100)
    assert getattr(o, how)(100) == 0
    assert pos_err(e.state()[0], o.state()[0], w.box) < 1e-6
    Tg, To = [], []
    kT = 3 * w.n * 0.0019872042586
    for k in range(9):
        getattr(e, how)(100)
        assert getattr(o, how)(100) == 0
        if k >= 1:
            Tg.append(e.observables()["temperature"])
            vo = o.state()[1]
            To.append((w.mass[:, None] * vo * vo).sum() / 418.4 / kT)
    assert abs(np.mean(Tg) / np.mean(To) - 1) < 0.04, (np.mean(Tg), np.mean(To))
    ob, c = e.observables(), o.counters()
    assert ob["error_flags"] == 0 and ob["step"] == 1000
    if how == "jump":
        for got, ref in ((ob["jump_proposals"], c[0]), (ob["jump_accepts"], c[1])):
            assert abs(got / ref - 1) < 0.02, (got, ref)


def _rdf_oo(frames, box, rmax=9.0, dr=0.05):
    from scipy.spatial import cKDTree
    edges = np.arange(0.0, rmax + dr, dr)
    h = np.zeros(len(edges) - 1)
    n_o = frames[0].shape[0] // 3
    for x in frames:
        o = np.mod(x[::3], box)
        p = cKDTree(o, boxsize=box).query_pairs(rmax, output_type="ndarray")
        d = o[p[:, 0]] - o[p[:, 1]]
        d -= box * np.round(d / box)
        h += np.histogram(np.sqrt((d * d).sum(1)), edges)[0]
    shell = 4.0 / 3.0 * np.pi * (edges[1:] ** 3 - edges[:-1] ** 3)
    ideal = shell * n_o / box ** 3 * n_o / 2 * len(frames)
    return h / ideal, dr, rmax


def _diffusion_groups(U, every_fs, groups=8):
    """D (1e-5 cm^2/s) of each of `groups` interleaved subsets of the oxygens
    from their unwrapped positions U[frame, oxygen, 3]: Einstein MSD over all
    time origins, linear fit over 20-80 % of the lags"""
    nt = U.shape[0]
    lags = np.arange(1, nt)
    t = lags * every_fs * 1e-3
    sel = (lags >= 0.2 * (nt - 1)) & (lags <= 0.8 * (nt - 1))
    out = []
    for g in range(groups):
        X = U[:, g::groups]
        msd = np.array([((X[l:] - X[:-l]) ** 2).sum(-1).mean() for l in lags])
        out.append(np.polyfit(t[sel], msd[sel], 1)[0] / 6.0 * 10.0)
    return np.array(out)


@pytest.mark.slow
@pytest.mark.parametrize("how", ["baoab", "jump", "jump_respa1_ewald"])
def test_mixed_precision_long_run_observables(M, how):
    """24,000-atom water from one equilibrated state in mixed precision and in
    FP64 (the FP64 mode follows the oracle event for event; the oracle itself
    cannot run this long at this size): mean temperature within 0.5 %, O-O
    radial distribution L1 distance <= 1e-2, and the oxygen self-diffusion
    within 5 %. D is estimated on eight interleaved groups of oxygens; the
    window (3000 fs, 9000 fs for JUMP under DSF, whose jumps damp diffusion)
    is long enough that the standard error of the FP64 estimate is below 2 %."""
    from paper_2412_15073_gb300 import systems
    w = systems.water_box(8000, box=62.1, seed=0)
    p = dict(PARAMS, skin=0.5, skin_outer=1.5)
    eq = M.Engine(precision=1, seed=31)
    eq.set_system(0, w, **(p | {"gamma": 20.0}))
    eq.baoab(500)
    w.x, w.v = eq.state()[0], eq.state()[1]
    eq.close()
    res = {}
    every, steps = 150, 3000
    if how == "jump":
        steps = 9000
    if how == "jump_respa1_ewald":
        # the paper's 96,000-atom settings (one ring, LJ long part at the outer level), 1:2:6 fs
        p = p | dict(dsf_alpha=0.42, coulomb_mode=1, pme_order=6, pme_spacing=0.8, r_split=6.0,
                     ring_r=[], lj_long_mode=2, skin=0.4, eps0=2.0)
        every = 144
    for prec in (0, 1):
        e = M.Engine(precision=prec, seed=32)
        e.set_system(0, w, **p)
        fn = (lambda k, e=e: e.jump_respa1(k // 6, 1.0, 2, 3)) if how == "jump_respa1_ewald" else getattr(e, how)
        T, frames, U = [], [], []
        for k in range(steps // every + 1):
            x, _, img, _ = e.state()
            frames.append(x)
            U.append((x + img * w.box)[::3])
            if k < steps // every:
                fn(every)
                T.append(e.observables()["temperature"])
        Dg = _diffusion_groups(np.stack(U), every)
        res[prec] = (np.mean(T), _rdf_oo(frames[1::2], w.box), Dg.mean(), Dg.std(ddof=1) / np.sqrt(len(Dg)))
        e.close()
    (T64, (g64, dr, rmax), D64, se64), (T32, (g32, _, _), D32, se32) = res[0], res[1]
    l1 = np.abs(g32 - g64).sum() * dr / rmax
    print(f"{how}: T {T32:.2f} vs {T64:.2f} K, RDF L1 {l1:.2e}, D {D32:.4f} +- {se32:.4f} vs "
          f"{D64:.4f} +- {se64:.4f} (1e-5 cm^2/s)")
    assert abs(T32 / T64 - 1) < 0.005
    assert l1 <= 1e-2
    assert se64 / D64 < 0.02, (se64, D64)
    assert abs(D32 / D64 - 1) < 0.05
