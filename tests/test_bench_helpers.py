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
    sample of the benchmark step): one JSON line whose value, ms_per_step,
    cpu_baseline and e2e agree"""
    import argparse
    import json

    bench.run_reference(argparse.Namespace(steps=1, warmup=0))
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "ns/day" and d["metric"] == bench.METRIC
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert abs(bench.ns_per_day(bench.DT_FS, d["ms_per_step"] * 1e-3) / d["value"] - 1) < 1e-9
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and "96,000" in d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "ns/day", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_pair_roofline_arithmetic():
    """52 FLOPs per pair over the mean time of one evaluation, against
    152 SMs x 128 lanes x 2 x clock"""
    r = bench.pair_roofline(ms_total=40.0, groups=100, pairs=20e6, clock_mhz=2000.0)
    assert r["ms_per_launch"] == 0.4
    assert abs(r["achieved"] - 52 * 20e6 / 0.4e-3 / 1e12) < 1e-12
    assert abs(r["peak"] - 152 * 128 * 2 * 2e9 / 1e12) < 1e-9
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-15 and r["unit"] == "TFLOP/s"
