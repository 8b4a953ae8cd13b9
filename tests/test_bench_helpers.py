"""Host-side helpers of bench.py that need no GPU: the diffusion estimate."""
import numpy as np

import bench


class FakeEngine:
    """Brownian walkers in a periodic box, wrapped like the engine wraps
    positions (x in [0, L), image counts in img)."""

    def __init__(self, n, box, D, dt_fs, seed=0):
        self.rng = np.random.default_rng(seed)
        self.box, self.D, self.dt = box, D, dt_fs * 1e-3
        self.u = self.rng.uniform(0, box, size=(n, 3))          # unwrapped

    def step(self, k):
        self.u += self.rng.normal(scale=np.sqrt(2 * self.D * self.dt * k), size=self.u.shape)

    def state(self):
        img = np.floor(self.u / self.box).astype(np.int32)
        x = self.u - img * self.box
        return x, np.zeros_like(x), img, x


def test_diffusion_estimate_recovers_brownian_D():
    D = 0.25                                                    # A^2/ps = 2.5e-5 cm^2/s
    e = FakeEngine(3 * 4000, 20.0, D, 1.0)
    got = bench.diffusion(e, e.step, 2000, 100, 20.0, 1.0)
    assert abs(got / 2.5 - 1) < 0.05, got


def test_diffusion_block_standard_error_covers_the_estimate():
    """the block standard error of D (four consecutive time blocks) is of the
    size of the spread of D over independent walks of the same length"""
    D = 0.25
    est, ses = [], []
    for seed in range(6):
        e = FakeEngine(3 * 600, 20.0, D, 1.0, seed=seed)
        d, _, se = bench.diffusion(e, e.step, 4000, 100, 20.0, 1.0, mass=np.ones(3 * 600), se=True)
        est.append(d)
        ses.append(se)
    spread = np.std(est, ddof=1)
    assert 0.3 < np.mean(ses) / spread < 3.0, (np.mean(ses), spread)
    assert abs(np.mean(est) / 2.5 - 1) < 0.05


def test_oxygen_rdf_of_an_ideal_gas_is_one():
    """_rdf_oo of uniformly scattered points (every third atom an 'oxygen')
    is 1 within its counting noise from 3 to 9 A"""
    rng = np.random.default_rng(4)
    frames = [rng.uniform(0, 40.0, size=(3 * 3000, 3)) for _ in range(4)]
    g, dr, rmax = bench._rdf_oo(frames, 40.0)
    r = (np.arange(len(g)) + 0.5) * dr
    sel = (r > 3.0) & (r < rmax)
    assert abs(g[sel].mean() - 1.0) < 0.02, g[sel].mean()


def test_bench_functions_name_only_defined_globals():
    """every global a function of bench.py reads exists (a deleted constant
    would otherwise only show on the GPU machine)"""
    import builtins
    import inspect
    import types

    import bench

    def code_objects(co):
        yield co
        for c in co.co_consts:
            if isinstance(c, types.CodeType):
                yield from code_objects(c)

    missing = set()
    for name, fn in inspect.getmembers(bench, inspect.isfunction):
        if fn.__module__ != "bench":
            continue
        for co in code_objects(fn.__code__):
            for g in co.co_names:
                if not hasattr(bench, g) and not hasattr(builtins, g):
                    # attribute names appear in co_names too: keep only names used as globals
                    if any(ins.opname in ("LOAD_GLOBAL", "LOAD_NAME") and ins.argval == g
                           for ins in __import__("dis").get_instructions(co)):
                        missing.add((name, g))
    assert not missing, missing


def test_reference_arm_prints_one_consistent_line(capsys):
    """bench.py --impl reference (the oracle on the host cores, a bounded
    sample of the benchmark cycle, here on a 1,536-atom box): one JSON line
    whose value, extrapolated cycle time, cpu_baseline and e2e agree, and
    whose steps x ms_per_step is the work it really did"""
    import argparse
    import json

    bench.run_reference(argparse.Namespace(steps=2, warmup=0, ref_mol=512))
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "ns/day" and d["metric"] == bench.METRIC
    assert d["value"] > 0 and d["higher_is_better"] is True
    full = d["ms_per_full_step_extrapolated"] * 1e-3
    assert abs(bench.ns_per_day(bench.CYCLE_FS, full) / d["value"] - 1) < 1e-9
    assert d["steps"] * d["ms_per_step"] * 1e-3 <= d["wall_s"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and "1,536" in d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "ns/day", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_roofline_arithmetic():
    """pair kernel: 52 FLOPs per pair over the mean time of one evaluation,
    against SMs x 128 lanes x 2 x clock; C' kernel: 20 B per proposal and
    128 B per atom over the mean launch time, against the HBM peak"""
    r = bench.pair_roofline(ms_total=40.0, groups=100, pairs=20e6, sms=148, clock_mhz=2000.0)
    assert r["ms_per_launch"] == 0.4
    assert abs(r["achieved"] - 52 * 20e6 / 0.4e-3 / 1e12) < 1e-12
    assert abs(r["peak"] - 148 * 128 * 2 * 2e9 / 1e12) < 1e-9
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-15 and r["unit"] == "TFLOP/s"
    c = bench.cphase_roofline(ms_total=10.0, groups=20, proposals=2e8, atoms=96000, hbm_gbs=6000.0, sms=152,
                              clock_mhz=1500.0, peak_kind="measured")
    nbytes = 20 * 1e7 + 128 * 96000
    assert abs(c["achieved"] - nbytes / 0.5e-3 / 1e9) < 1e-9 and c["unit"] == "GB/s"
    assert abs(c["frac"] - c["achieved"] / 6000.0) < 1e-15
    assert abs(c["issue_view"]["peak"] - 152 * 4 * 32 * 1.5e9 / 1e12) < 1e-9


def test_matched_flags_and_best_pair():
    """matched: mean T within 0.5 % and D within 5 % of the reference; the
    fastest matched run of each family and their ratio"""
    ref = {"D": 2.0, "T_mean": 300.0}
    runs = {"jump_a": {"ns_per_day": 200.0, "D": 2.08, "T_mean": 301.0},
            "jump_b": {"ns_per_day": 250.0, "D": 2.2, "T_mean": 300.0},
            "baoab_a": {"ns_per_day": 180.0, "D": 1.95, "T_mean": 299.0},
            "baoab_b": {"ns_per_day": 190.0, "D": 2.0, "T_mean": 302.0}}
    for v in runs.values():
        bench.matched_flags(v, ref)
    assert [runs[k]["matched"] for k in ("jump_a", "jump_b", "baoab_a", "baoab_b")] == [True, False, True, False]
    b = bench.best_matched(runs)
    assert b["jump"]["run"] == "jump_a" and b["baoab"]["run"] == "baoab_a"
    assert abs(b["jump_over_baoab"] - 200.0 / 180.0) < 1e-12
