"""Throughput of the JUMP path against the GPU's own BAOAB path at matched
temperature and diffusion constant.

Headline workload (96,000 atoms): 32,000 flexible 3-site waters in a 98.6 A
periodic cube, 300 K, gamma = 1/ps, mixed precision (FP32 pair math, 64-bit
fixed-point sums, FP64 integration). JUMP-RESPA1 against BAOAB-RESPA1, three
levels: delta = 1 fs (bonded terms), kappa = 2 fs (short-range pairs; the
jumps of JUMP-RESPA1), Delta = 4 fs (the slow level). Electrostatics as in the
paper's runs: Ewald real space erfc(a r)/r to r_E = 10 A with a = 0.42/A,
smooth PME of order 6 on a 0.8 A grid (125^3), short-range split r_c = 6 A
(switch width 0.5 A). JUMP-RESPA1 jumps the (1 - chi) real-space Coulomb part
(adaptive eps0 = 2, one ring) and keeps the (1 - chi) LJ part deterministic at
the slow level with the reciprocal sum; BAOAB-RESPA1 evaluates the (1 - chi)
pairs there. A step is one outer cycle (4 fs). Both runs are matched against
plain BAOAB at 1 fs (mean temperature within 0.5 %, oxygen self-diffusion
within 5 %) on the same equilibrated start.

The DSF form of the same water (r_c 5 A, DSF 0.2/A, JUMP at 1 fs with rings at
5.25/6/7.5 A, eps0 0.1) is reported beside it: there the jumps damp diffusion
(`--only dsf_sweep` sweeps r_c and eps0), so it has no matched setting.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line. Under torchrun (N > 1) every rank advances its own
replica (replicas only: the path has no exchange step) and rank 0 prints.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_MOL, BOX = 32000, 98.6
DT_FS = 1.0
# DSF water: the specified electrostatics (damped shifted force Coulomb)
DSF = dict(r_cut=10.0, r_split=5.0, h_switch=0.5, r_mid=5.5, dsf_alpha=0.2, gamma=1.0,
           temperature=300.0, eps0=0.1, eps_mode=1, skin=0.5, skin_outer=1.5)
# list parameters tuned per integrator (both measured on this workload): JUMP
# takes four rings (edges r_c - h, 5.25, 6, 7.5, r_E) and a 0.3 A skin, since
# every ring partner in the skin is a proposal that is always rejected; BAOAB
# the 0.5 A skin that minimises its pair-force plus rebuild time
DSF_JUMP = DSF | dict(ring_r=[5.25, 6.0, 7.5], skin=0.3)
DSF_BAOAB = DSF
# Ewald water (the paper's electrostatics and 96,000-atom JUMP settings). With
# weak jumped forces the proposal count is set by the 1/eps0 floor, not by the
# ring bounds: one ring, fewer list kinds; a 0.4 A skin for both (the fastest
# of 0.3 - 0.8 A for each integrator, --only skin_sweep)
EWALD = dict(dsf_alpha=0.42, coulomb_mode=1, pme_order=6, pme_spacing=0.8, r_split=6.0)
EW_JUMP = DSF_JUMP | EWALD | dict(ring_r=[], lj_long_mode=2, skin=0.4, eps0=2.0)
EW_BAOAB = DSF_BAOAB | EWALD | dict(skin=0.4)     # the measured best skin of BAOAB-RESPA1 (--only skin_sweep)
M_MID, N_OUT = 2, 2                       # kappa = 2 delta, Delta = 2 kappa
CYCLE_FS = M_MID * N_OUT * DT_FS          # one headline step
EW_WINDOW_FS = 480                        # timing window of the Ewald comparison runs
DSF_WINDOW = 200                          # timing window (steps) of the DSF runs
METRIC = "ns/day & Gpair-evals/s, JUMP vs BAOAB on 1 GB300 at matched T/D (97k atoms)"
WORKLOAD = ("water 96,000 atoms (32,000 flexible 3-site waters, 98.6 A cube), Ewald a 0.42/A real space to "
            "10 A + smooth PME (order 6, 125^3), split r_c 6 A; JUMP-RESPA1 (eps0 2, one ring, LJ long part at "
            "the slow level) vs BAOAB-RESPA1, delta 1 / kappa 2 / Delta 4 fs, 300 K, gamma 1/ps; step = one 4 fs cycle")
DSF_WORKLOAD = ("water 96,000 atoms, LJ + DSF 0.2/A to 10 A, r_c 5 A, rings at 5.25/6/7.5 A, adaptive eps0 0.1; "
                "JUMP 1 fs vs BAOAB 1 fs")
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
CLASSES = ["pair_force", "bonded", "velocity_phase", "kick_aoa", "list_cells_outer", "bookkeeping",
           "ewald_recip", "list_inner", "rate_order"]
# FP32 work of one pair of the pair kernel (min image, r^2, erfc/exp, DSF, LJ,
# switch, fixed point), counted from the kernel source
FLOP_PER_PAIR = 52
# algorithmic HBM bytes of the C' kernel: per proposal the partner's list
# entry (4 B) and its scaled position and charge (16 B); per atom and launch
# its velocity (read and written, 48 B), acceleration (24 B), own position
# (16 B), ring bounds (16 B), ring counts (16 B) and reduced mass (8 B)
CPHASE_BYTES_PER_PROPOSAL = 20
CPHASE_BYTES_PER_ATOM = 128
# executed thread-instructions per C' proposal: one ncu capture (--set full) of
# a single-phase launch of the DSF workload executed 148.3 M warp instructions
# with 13.7 lanes active on average for 3.574 M proposals
CPHASE_INST_PER_PROPOSAL = 148.3e6 * 13.7 / 3.574e6
# algorithmic bytes of the inner list filter: per outer candidate its entry
# (4 B), per kept entry its store (4 B), per atom its position (16 B) and the
# counts of the list kinds it fills (4 B each, three kinds)
INNER_BYTES_PER_CAND = 4
INNER_BYTES_PER_ENTRY = 4
INNER_BYTES_PER_ATOM = 16 + 12
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) that one ncu
# capture measured for one rebuild launch of k_inner_lists<69> (short list, one
# ring, LJ list) on the headline workload, before the kernel gained its exit
# for launches without a rebuild; reported beside a null traffic until the
# capture is taken again
INNER_TRAFFIC_NCU_EARLIER = 265.834e6 + 183.101e6


def ns_per_day(fs_simulated: float, seconds: float) -> float:
    return fs_simulated * 1e-6 / seconds * 86400.0


def peaks():
    try:
        return json.load(open(PEAKS)), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def pair_roofline(ms_total: float, groups: int, pairs: float, sms: int, clock_mhz: float) -> dict:
    """FP32 roofline of the pair kernel of one BAOAB force evaluation: the
    algorithmic FLOPs (FLOP_PER_PAIR per unique pair within the cutoff) over
    the mean device time of one evaluation (CUDA events of the library's
    pair-force class) against SMs x 128 lanes x 2 x the SM clock."""
    per_launch_s = ms_total / max(groups, 1) * 1e-3
    achieved = FLOP_PER_PAIR * pairs / per_launch_s / 1e12
    peak = sms * 128 * 2 * clock_mhz * 1e6 / 1e12
    return {"bound": "fp32", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "kernel": "k_force (BAOAB full pairs)", "units_per_launch": pairs,
            "ops_per_unit": FLOP_PER_PAIR, "ms_per_launch": per_launch_s * 1e3,
            "peak_source": f"FP32: {sms} SMs x 128 lanes x 2 x {clock_mhz:.0f} MHz (median SM clock sampled "
                           f"while the bench ran)"}


def cphase_roofline(ms_total, groups, proposals, atoms, hbm_gbs, sms, clock_mhz, peak_kind):
    """HBM roofline of the C' kernel (the velocity phase of the JUMP step):
    algorithmic bytes per launch over its mean device time, against the
    measured copy bandwidth; beside it the issue rate implied by the executed
    instructions per proposal (from an ncu capture) against SMs x 4 schedulers
    x 32 lanes x the SM clock."""
    per_launch_s = ms_total / max(groups, 1) * 1e-3
    props = proposals / max(groups, 1)
    nbytes = CPHASE_BYTES_PER_PROPOSAL * props + CPHASE_BYTES_PER_ATOM * atoms
    achieved = nbytes / per_launch_s / 1e9
    issue = CPHASE_INST_PER_PROPOSAL * props / per_launch_s / 1e12
    issue_peak = sms * 4 * 32 * clock_mhz * 1e6 / 1e12
    return {"bound": "hbm", "achieved": achieved, "peak": hbm_gbs, "unit": "GB/s", "frac": achieved / hbm_gbs,
            "traffic": None, "kernel": "k_cphase_f (C' pair jumps and J' bounces, mixed)",
            "bytes_per_launch": nbytes, "proposals_per_launch": props, "atoms": atoms,
            "bytes_model": f"{CPHASE_BYTES_PER_PROPOSAL} B per proposal + {CPHASE_BYTES_PER_ATOM} B per atom",
            "ms_per_launch": per_launch_s * 1e3, "peak_kind": peak_kind,
            "issue_view": {"achieved": issue, "peak": issue_peak, "unit": "T thread-instructions/s",
                           "frac": issue / issue_peak, "inst_per_proposal": CPHASE_INST_PER_PROPOSAL,
                           "peak_source": f"{sms} SMs x 4 x 32 lanes x {clock_mhz:.0f} MHz"}}


class Clocks:
    """nvidia-smi samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.out = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # the timed region starts once the sampler is running (its first line is out)
            t0 = time.time()
            while not self.out and time.time() - t0 < 5.0 and self.proc.poll() is None:
                time.sleep(0.01)
            self.n0 = len(self.out)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.out.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        # the lines written after the timed region began (the first one may predate it)
        for line in self.out[getattr(self, "n0", 0):] or self.out:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def pair_counts(x, box, r, n_mol_atoms=3):
    """Unique intermolecular pairs within r (periodic cKDTree)."""
    from scipy.spatial import cKDTree
    t = cKDTree(np.mod(x, box), boxsize=box)
    pairs = t.query_pairs(r, output_type="ndarray")
    same = (pairs[:, 0] // n_mol_atoms) == (pairs[:, 1] // n_mol_atoms)
    return int((~same).sum())


def _einstein_D(X, every, dt_fs):
    """D (1e-5 cm^2/s) from unwrapped positions X[t, atom, 3] sampled every `every` steps"""
    nt = X.shape[0]
    lags = np.arange(1, nt)
    msd = np.array([((X[l:] - X[:-l]) ** 2).sum(-1).mean() for l in lags])
    t = lags * every * dt_fs * 1e-3                     # ps
    sel = (lags >= 0.2 * (nt - 1)) & (lags <= 0.8 * (nt - 1))
    slope = np.polyfit(t[sel], msd[sel], 1)[0]          # A^2 / ps
    return slope / 6.0 * 10.0                           # A^2/ps = 1e-4 cm^2/s -> units of 1e-5 cm^2/s


def diffusion(e, integ, steps, every, box, dt_fs, mass=None, replica=0, se=False):
    """Self-diffusion constant of the oxygens (atoms 0, 3, 6, ...) from the
    Einstein relation: MSD of the unwrapped positions over all time origins,
    slope of a linear fit over 20-80 % of the lag window, D = slope / 6.
    Returns D in 1e-5 cm^2/s; with the masses (amu), (D, mean temperature over
    the same samples, 3N degrees of freedom); with se, also a standard error
    of D from four consecutive time blocks of the window (D of each block,
    their spread over sqrt(4)), which also holds the slow, collective part
    of the fluctuations that a split of the oxygens into groups misses."""
    xs, ts = [], []
    for k in range(steps // every + 1):
        x, v, img, _ = e.state(replica) if replica else e.state()
        xs.append((x + img * box)[::3])
        if mass is not None:
            ts.append((mass[:, None] * v * v).sum() / (3 * len(mass) * 0.0019872041 * 418.4))
        if k < steps // every:
            integ(every)
    X = np.stack(xs)
    D = _einstein_D(X, every, dt_fs)
    if mass is None:
        return D
    if not se:
        return D, float(np.mean(ts))
    nb = X.shape[0] // 4
    Db = np.array([_einstein_D(X[b * nb:(b + 1) * nb + 1], every, dt_fs) for b in range(4)])
    return D, float(np.mean(ts)), float(Db.std(ddof=1) / np.sqrt(4))


def matched_flags(run: dict, ref: dict) -> None:
    """matched against the reference dynamics: mean T within 0.5 %, D within 5 %"""
    if run.get("D") and ref.get("D") and ref.get("T_mean"):
        run["D_ratio"] = run["D"] / ref["D"]
        run["T_ratio"] = run["T_mean"] / ref["T_mean"]
        if run.get("D_se") is not None and ref.get("D_se") is not None:
            # standard error of the ratio (the two runs are independent)
            run["D_ratio_se"] = run["D_ratio"] * float(np.hypot(run["D_se"] / run["D"], ref["D_se"] / ref["D"]))
        run["matched"] = bool(abs(run["D_ratio"] - 1) <= 0.05 and abs(run["T_ratio"] - 1) <= 0.005)


def best_matched(res: dict) -> dict:
    """fastest matched run of each family and the ratio of the two"""
    best = {}
    for fam in ("jump", "baoab"):
        cands = [(k, v) for k, v in res.items() if isinstance(v, dict) and k.startswith(fam) and v.get("matched")]
        if cands:
            k, v = max(cands, key=lambda kv: kv[1]["ns_per_day"])
            best[fam] = {"run": k, "ns_per_day": v["ns_per_day"], "D_ratio": v.get("D_ratio"),
                         "T_ratio": v.get("T_ratio")}
    if len(best) == 2:
        best["jump_over_baoab"] = best["jump"]["ns_per_day"] / best["baoab"]["ns_per_day"]
    return best


# ---------------------------------------------------------------- CPU oracle
def oracle_cycle_cost(sys_, params, mode, n_grad, n_phase, n_bonded, n_recip, tau2, runs, seed=0):
    """Time the FP64 oracle on a bounded sample of one step of the workload.
    The O(N^2) per-atom part (n_grad brute-force nonbonded gradients and
    n_phase C' phases, each followed by J' when LJ jumps) runs for lists of
    atoms drawn at random; the whole-system parts (n_bonded bonded gradients,
    n_recip smooth-PME sums) are timed once. runs: (atoms per sample, samples,
    OpenMP threads, 0 = all) per configuration. Returns, per configuration,
    (seconds of one full step, threads used, seconds of each sampled step), and
    the seconds of the whole-system parts."""
    import oracle
    oracle.build()
    o = oracle.Oracle(sys_, seed=seed, **params)
    rng = np.random.default_rng(seed)
    t0 = time.perf_counter()
    for _ in range(n_bonded):
        o.gradient(oracle.GRAD_BONDED)
    for _ in range(n_recip):
        o.ewald_recip_pme()
    t_global = time.perf_counter() - t0
    out = []
    for n_at, n_samples, nthreads in runs:
        per, thr = [], 1
        for s_idx in range(n_samples):
            atoms = rng.choice(sys_.n, n_at, replace=False)
            t1 = time.perf_counter()
            thr = o.sample_atom_work(atoms, mode, n_grad, n_phase, tau2, s_idx, nthreads)
            per.append(time.perf_counter() - t1)
        out.append((t_global + sys_.n * sum(per) / (n_at * n_samples), thr, per))
    return out, t_global


def headline_oracle_cost(sys_, runs):
    """One JUMP-RESPA1 cycle (1:2:4 fs) of the headline workload on the
    oracle: per atom two short-range gradients (one per kappa step), the
    (1 - chi) LJ part of the slow level (one more brute-force pass) and four
    C' phases (two per kappa step); whole system four bonded gradients (one
    per delta step) and one smooth-PME sum (the slow level)."""
    return oracle_cycle_cost(sys_, EW_JUMP, 3, 3, 4, 4, 1, M_MID * DT_FS * 0.5e-3, runs)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2412_15073_gb300 import systems
    n_mol = getattr(args, "ref_mol", N_MOL)
    w = systems.water_box(n_mol, box=(n_mol / 32000) ** (1 / 3) * BOX, seed=0)
    n_sample = 64
    import oracle
    oracle.build()
    t_start = time.perf_counter()
    (res, t_global) = headline_oracle_cost(w, [(n_sample, args.warmup + args.steps, 0)])
    t_cycle, thr, per = res[0]
    timed = per[args.warmup:]
    secs = sum(timed)
    steps_equiv = len(timed) * n_sample / w.n
    # one full cycle: the whole-system parts once plus every atom's share
    value = ns_per_day(CYCLE_FS, t_cycle)
    sample = (f"per step: {n_sample} of {w.n:,} atoms, each with its per-atom work of one JUMP-RESPA1 cycle "
              f"(three O(N) nonbonded passes, four C' phases) on {thr} threads; the whole-system parts (four "
              f"bonded gradients, one smooth-PME sum: {t_global:.1f} s) timed once and added; list builds "
              f"excluded; value extrapolated to the full cycle")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "ns/day", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup,
            # the wall time of each sampled step (what this run did), and the full cycle it stands for
            "ms_per_step": secs / max(len(timed), 1) * 1e3,
            "ms_per_full_step_extrapolated": t_cycle * 1e3, "full_steps_equivalent": steps_equiv,
            "wall_s": time.perf_counter() - t_start,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD if n_mol == N_MOL else f"{w.n} atoms (test)",
                                            "parallelism": "replicas"},
            "cpu_baseline": {"value": value, "unit": "ns/day", "cores": thr, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "ns/day", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- multi-rank
class Ranks:
    """Ranks of a multi-GPU run (one process per GPU, RANK / WORLD_SIZE /
    LOCAL_RANK from the launcher). Each rank advances its own replica: there is
    no data-path collective, only a barrier around the timed region and the
    maximum of the measured times over ranks."""

    def __init__(self, backend="nccl"):
        import torch
        self.torch = torch
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.cuda = backend == "nccl"
        self.dist = None
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend)
            self.dist = dist

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()
        if self.cuda:
            self.torch.cuda.synchronize()

    def max(self, x: float) -> float:
        if self.dist is None:
            return x
        t = self.torch.tensor([x], dtype=self.torch.float64, device="cuda" if self.cuda else "cpu")
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def seed(self, base: int) -> int:
        """Philox seed of this rank's replica."""
        return base + 1000 * self.rank

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()


def timed(fn, steps, stream):
    """device time of fn(steps) by CUDA events on the library's stream"""
    import torch
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def profiled(e, fn, steps):
    """per-class device time (ms), timed groups and kernels of fn(steps), plain launches"""
    e.profile(enable=1, reset=True)
    try:
        fn(steps)
    finally:
        ms, groups, _ = e.profile(enable=0)
    return ms, groups


def e2e_run(e, run, args, M, torch, n, world, max_over_ranks, barrier, fs_per_step):
    """Same metric through the public C ABI with pinned host buffers: per bench
    step (K steps) md_set_state from host, the integrator call, md_get_state to host."""
    x, v, img, xb, xo = e.state(outer=True)
    step0 = e.observables()["step"]
    hx = [torch.from_numpy(a).pin_memory().numpy() for a in (x, v, xb, xo)]
    himg = torch.from_numpy(img).pin_memory().numpy()
    barrier()
    t0 = time.perf_counter()
    e.set_state(0, hx[0], hx[1], himg, hx[2], hx[3], step=step0)
    run(args.steps)
    e._ck(e.L.md_get_state(e.h, 0, M._ptr(hx[0]), M._ptr(hx[1]), M._ptr(himg), M._ptr(hx[2]), M._ptr(hx[3])))
    torch.cuda.synchronize()
    t = max_over_ranks(time.perf_counter() - t0)
    state_bytes = n * (4 * 3 * 8 + 3 * 4)
    # one round trip of the whole state per call of K steps: per step that is state_bytes / K
    return {"value": ns_per_day(world * args.steps * fs_per_step, t), "unit": "ns/day",
            "h2d_bytes_per_step": state_bytes / args.steps, "d2h_bytes_per_step": state_bytes / args.steps,
            "bytes_per_round_trip": state_bytes, "steps_per_round_trip": args.steps,
            "path": "md_set_state(pinned host) + md_step_jump_respa1(K cycles) + md_get_state(pinned host)"}


def relax(M, w, params, steps, seed, device, stream, max_replicas=1, systems_=None, gamma=20.0, dt_fs=1.0):
    """BAOAB at strong friction (gamma, 1/ps) from the given start: positions
    and velocities are written back into the system(s)"""
    syss = systems_ or [w]
    eq = M.Engine(precision=M.MD_MIXED, seed=seed, device=device, stream=stream.cuda_stream,
                  max_replicas=max(max_replicas, len(syss)))
    for r, s in enumerate(syss):
        eq.set_system(r, s, **(params | {"gamma": gamma}))
    eq.baoab(max(steps, 1), dt_fs)
    for r, s in enumerate(syss):
        s.x, s.v = eq.state(r)[0], eq.state(r)[1]
    eq.close()


# ---------------------------------------------------------------- legs
def ewald_runs(args, M, engine, stream, world, max_over_ranks, barrier, mass, box=BOX, d_fs=None, names=None):
    """Ewald comparison on one equilibrated start: ns/day over a fixed window
    (EW_WINDOW_FS, independent of --steps), per-class device time, and the
    mean temperature and oxygen self-diffusion of each run, matched against
    plain BAOAB at 1 fs. Runs: JUMP-RESPA1 and BAOAB-RESPA1 at Delta = 4 fs
    (the headline) and 6 fs (the paper's 1:2:6)."""
    d_fs = args.dwindow if d_fs is None else d_fs
    runs = [("baoab_1fs", 4, "baoab", 1, 1, EW_BAOAB),
            ("jump_respa1_D4", 5, "jump_respa1", 2, 2, EW_JUMP),
            ("baoab_respa1_D4", 6, "baoab_respa1", 2, 2, EW_BAOAB),
            ("jump_respa1_D6", 5, "jump_respa1", 2, 3, EW_JUMP),
            ("baoab_respa1_D6", 6, "baoab_respa1", 2, 3, EW_BAOAB)]
    if names:
        runs = [r for r in runs if r[0] in names or r[0] == "baoab_1fs"]
    res = {}
    for name, seed, meth, m_mid, n_out, params in runs:
        per_cycle = m_mid * n_out
        e = engine(seed, params)
        run = (lambda k, e=e: e.baoab(k)) if meth == "baoab" else \
            (lambda k, e=e, meth=meth, m=m_mid, q=n_out: getattr(e, meth)(k, 1.0, m, q))
        try:
            run(max(1, 120 // per_cycle))           # settle in the Ewald force field (and capture graphs)
            cyc = max(EW_WINDOW_FS // per_cycle, 1)
            c0 = e.observables()
            barrier()
            t = max_over_ranks(timed(run, cyc, stream))
            c1 = e.observables()
            r = {"ns_per_day": ns_per_day(world * cyc * per_cycle * DT_FS, t),
                 "ms_per_fs": t / (cyc * per_cycle) * 1e3, "fs_timed": cyc * per_cycle, "T": c1["temperature"],
                 "stable": bool(abs(c1["temperature"] / 300.0 - 1) < 0.1)}
            if meth == "jump_respa1":
                r["proposals_per_atom_fs"] = (c1["jump_proposals"] - c0["jump_proposals"]) / (e.n[0] * cyc * per_cycle)
            pc = max(1, 240 // per_cycle)
            ms, _ = profiled(e, run, pc)
            r["class_ms_per_fs"] = {c: round(float(m) / (pc * per_cycle), 4) for c, m in zip(CLASSES, ms)}
            if d_fs > 0 and r["stable"]:
                every = 96 if d_fs >= 960 else 24       # a multiple of every cycle length (1, 4, 6 fs)
                nd = d_fs // every * every
                r["D"], r["T_mean"], r["D_se"] = diffusion(e, lambda k: run(k // per_cycle), nd, every, box,
                                                           DT_FS, mass, se=True)
            res[name] = r
        except M.MDError as ex:
            res[name] = {"error": str(ex), "stable": False}
        e.close()
    ref = res.get("baoab_1fs", {})
    for k, v in res.items():
        if k != "baoab_1fs" and isinstance(v, dict) and "ns_per_day" in v:
            matched_flags(v, ref)
    res["best_matched"] = best_matched(res)
    res["D_unit"] = "1e-5 cm^2/s"
    res["D_window_ps"] = d_fs * 1e-3
    res["criterion"] = "matched: mean T within 0.5 % and D within 5 % of plain BAOAB at 1 fs"
    return res


def dsf_leg(args, M, engine, stream, world, max_over_ranks, barrier, mass, sms, clock_mhz, hbm, peak_kind):
    """DSF water: JUMP (1 fs) against BAOAB (1 fs) over a fixed window, with
    D and T of both, the roofline of the C' kernel of the JUMP step and of the
    pair kernel of the BAOAB step (profiled runs of their own)."""
    out = {"workload": DSF_WORKLOAD}
    ej = engine(1, DSF_JUMP)
    eb = engine(2, DSF_BAOAB)
    ej.jump(args.warmup)
    eb.baoab(args.warmup)
    c0 = ej.observables()
    barrier()
    tj = max_over_ranks(timed(ej.jump, DSF_WINDOW, stream))
    barrier()
    tb = max_over_ranks(timed(eb.baoab, DSF_WINDOW, stream))
    c1 = ej.observables()
    n = ej.n[0]
    out["jump_ns_per_day"] = ns_per_day(world * DSF_WINDOW * DT_FS, tj)
    out["baoab_ns_per_day"] = ns_per_day(world * DSF_WINDOW * DT_FS, tb)
    out["speed_ratio"] = out["jump_ns_per_day"] / out["baoab_ns_per_day"]
    out["steps_timed"] = DSF_WINDOW
    props = (c1["jump_proposals"] - c0["jump_proposals"] + c1["bps_proposals"] - c0["bps_proposals"]) / DSF_WINDOW
    pairs_short = pair_counts(ej.state()[0], BOX, DSF["r_split"])
    pairs_full = pair_counts(eb.state()[0], BOX, DSF["r_cut"])
    out["gpair_evals_per_s"] = {"jump": world * (pairs_short + props) * DSF_WINDOW / tj / 1e9,
                                "baoab": world * pairs_full * DSF_WINDOW / tb / 1e9}
    out["proposals_per_atom_step"] = (c1["jump_proposals"] - c0["jump_proposals"]) / (n * DSF_WINDOW)
    out["accept_frac"] = (c1["jump_accepts"] - c0["jump_accepts"]) / max(c1["jump_proposals"] - c0["jump_proposals"], 1)
    # C' kernel of the JUMP step
    cp0 = ej.observables()
    ms, groups = profiled(ej, ej.jump, 100)
    cp1 = ej.observables()
    k = CLASSES.index("velocity_phase")
    props_tot = (cp1["jump_proposals"] - cp0["jump_proposals"]) + (cp1["bps_proposals"] - cp0["bps_proposals"])
    out["roofline_cphase"] = cphase_roofline(float(ms[k]), int(groups[k]), props_tot, n, hbm, sms, clock_mhz,
                                             peak_kind)
    out["roofline_cphase"]["share_of_step"] = float(ms[k] / ms.sum())
    out["jump_class_ms_per_step"] = {c: round(float(m) / 100, 4) for c, m in zip(CLASSES, ms)}
    msb, gb = profiled(eb, eb.baoab, 100)
    out["pair_roofline"] = pair_roofline(float(msb[0]), int(gb[0]), pairs_full, sms, clock_mhz)
    out["baoab_class_ms_per_step"] = {c: round(float(m) / 100, 4) for c, m in zip(CLASSES, msb)}
    if args.dwindow > 0:
        nd = args.dwindow // 200 * 100          # half the Ewald window: D of JUMP here is far from BAOAB's
        jd, jt = diffusion(ej, ej.jump, nd, 100, BOX, DT_FS, mass)
        bd, bt = diffusion(eb, eb.baoab, nd, 100, BOX, DT_FS, mass)
        out["jump"] = {"ns_per_day": out["jump_ns_per_day"], "D": jd, "T_mean": jt}
        ref = {"D": bd, "T_mean": bt}
        matched_flags(out["jump"], ref)
        out["baoab"] = ref
        out["effective_jump_ns_per_day"] = out["jump_ns_per_day"] * jd / bd
        out["D_unit"] = "1e-5 cm^2/s"
        out["D_window_ps"] = nd * DT_FS * 1e-3
    ej.close()
    eb.close()
    return out


def dsf_sweep(args, M, engine, stream, mass):
    """DSF water at 1 fs: JUMP with the split radius r_c in {5, 6, 7} A (the
    rings move with it) and eps0 in {0.1, 1, 2} (adaptive), against BAOAB at
    1 fs: ns/day, proposals, D / D_BAOAB and T."""
    out = {"window_steps": DSF_WINDOW, "D_window_ps": args.dwindow * 1e-3}
    eb = engine(2, DSF_BAOAB)
    eb.baoab(20)
    tb = timed(eb.baoab, DSF_WINDOW, stream)
    bd, bt = diffusion(eb, eb.baoab, args.dwindow // 100 * 100, 100, BOX, DT_FS, mass)
    eb.close()
    out["baoab"] = {"ns_per_day": ns_per_day(DSF_WINDOW * DT_FS, tb), "D": bd, "T_mean": bt}
    for rc in args.sweep_rc:
        for eps0 in args.sweep_eps0:
            p = DSF_JUMP | {"r_split": rc, "ring_r": [rc - 0.25, rc + 0.5, rc + 2.0], "eps0": eps0}
            name = f"rc{rc:g}_eps{eps0:g}"
            e = engine(1, p)
            try:
                e.jump(20)
                c0 = e.observables()
                t = timed(e.jump, DSF_WINDOW, stream)
                c1 = e.observables()
                r = {"ns_per_day": ns_per_day(DSF_WINDOW * DT_FS, t),
                     "proposals_per_atom_step": (c1["jump_proposals"] - c0["jump_proposals"]) / (e.n[0] * DSF_WINDOW)}
                r["D"], r["T_mean"] = diffusion(e, e.jump, args.dwindow // 100 * 100, 100, BOX, DT_FS, mass)
                matched_flags(r, out["baoab"])
                r["speed_ratio"] = r["ns_per_day"] / out["baoab"]["ns_per_day"]
                out[name] = r
            except M.MDError as ex:
                out[name] = {"error": str(ex)}
            e.close()
    return out


def _rdf_oo(frames, box, rmax=9.0, dr=0.05):
    """O-O radial distribution over the frames (periodic cKDTree)"""
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
    return h / (shell * n_o / box ** 3 * n_o / 2 * len(frames)), dr, rmax


def precision_leg(args, M, stream, local):
    """The 24,000-atom water of the precision study (8,000 molecules, 62.1 A,
    DSF 0.2/A to 9 A, split 5 A): BAOAB, JUMP and JUMP-RESPA (1:2 fs) from
    one equilibrated state, each in FP64 and in mixed precision for the same
    number of steps; the error of each observable of the mixed run against
    the FP64 run (the FP64 mode follows the FP64 oracle event for event, which
    is too slow to run this long at this size): mean temperature, O-O radial
    distribution (L1 distance), oxygen self-diffusion, and the wall time."""
    from paper_2412_15073_gb300 import systems
    box = 62.1
    w = systems.water_box(8000, box=box, seed=0)
    p = dict(r_cut=9.0, r_split=5.0, h_switch=0.5, r_mid=5.5, dsf_alpha=0.2, gamma=1.0, temperature=300.0,
             eps0=0.1, eps_mode=1, skin=0.5, skin_outer=1.5)
    eq = M.Engine(precision=M.MD_MIXED, seed=31, device=local, stream=stream.cuda_stream)
    eq.set_system(0, w, **(p | {"gamma": 20.0}))
    eq.baoab(500)
    w.x, w.v = eq.state()[0], eq.state()[1]
    eq.close()
    steps, every = args.psteps // 150 * 150, 150
    out = {"workload": "water 24,000 atoms (8,000 flexible 3-site waters, 62.1 A), DSF 0.2/A to 9 A, split 5 A, "
                       "300 K, gamma 1/ps, 1 fs; JUMP-RESPA 1:2 fs", "steps": steps}
    runs = [("baoab", lambda e, k: e.baoab(k)), ("jump", lambda e, k: e.jump(k)),
            ("jump_respa", lambda e, k: e.jump_respa(k // 2, 1.0, 2))]
    for name, fn in runs:
        res = {}
        for prec in (M.MD_FP64, M.MD_MIXED):
            e = M.Engine(precision=prec, seed=32, device=local, stream=stream.cuda_stream)
            e.set_system(0, w, **p)
            T, frames, U = [], [], []
            t0 = time.perf_counter()
            for k in range(steps // every + 1):
                x, _, img, _ = e.state()
                frames.append(x)
                U.append((x + img * box)[::3])
                if k < steps // every:
                    fn(e, every)
                    T.append(e.observables()["temperature"])
            wall = time.perf_counter() - t0
            X = np.stack(U)
            D = _einstein_D(X, every, DT_FS)
            nb = X.shape[0] // 4
            Db = np.array([_einstein_D(X[b * nb:(b + 1) * nb + 1], every, DT_FS) for b in range(4)])
            res[prec] = (float(np.mean(T)), _rdf_oo(frames[1::2], box), D, float(Db.std(ddof=1) / 2), wall)
            e.close()
        (T64, (g64, dr, rmax), D64, se64, w64), (T32, (g32, _, _), D32, se32, w32) = res[M.MD_FP64], res[M.MD_MIXED]
        out[name] = {"T_fp64": T64, "T_mixed": T32, "T_rel_err": T32 / T64 - 1,
                     "rdf_L1": float(np.abs(g32 - g64).sum() * dr / rmax),
                     "D_fp64": D64, "D_fp64_se": se64, "D_mixed": D32, "D_mixed_se": se32, "D_rel_err": D32 / D64 - 1,
                     "wall_s_fp64": w64, "wall_s_mixed": w32}
    return out


def dsf_respa1(args, M, engine, stream, world, max_over_ranks, barrier):
    """DSF RESPA1 stability: delta 1, kappa 2, Delta 2/4/6 fs; the outer level
    of JUMP-RESPA1 is empty without a reciprocal part. A run whose temperature
    leaves 300 K by more than 10 % is reported as unstable."""
    out = {"levels": "delta 1 fs, kappa 2 fs, Delta 2/4/6 fs"}
    runs = [("jump_respa1", 3, "jump_respa1", 1)] + [(f"baoab_respa1_D{2 * q}", 4, "baoab_respa1", q)
                                                   for q in (1, 2, 3)]
    for name, seed, meth, n_out in runs:
        per_cycle = 2 * n_out
        cyc = max(DSF_WINDOW // per_cycle, 1)
        e = engine(seed, DSF_JUMP if meth.startswith("jump") else DSF_BAOAB)
        try:
            getattr(e, meth)(2, 1.0, 2, n_out)
            barrier()
            t = max_over_ranks(timed(lambda k: getattr(e, meth)(k, 1.0, 2, n_out), cyc, stream))
            T = e.observables()["temperature"]
            out[name] = {"ns_per_day": ns_per_day(world * cyc * per_cycle * DT_FS, t), "T": T,
                         "stable": bool(abs(T / 300.0 - 1) < 0.1)}
        except M.MDError as ex:
            out[name] = {"error": str(ex), "stable": False}
        e.close()
    return out


# the batched ensemble: 64 water boxes of 216-2,000 molecules (sizes from seed
# 1, each its own box and Philox stream)
ENSEMBLE_DSF = dict(r_cut=9.0, r_split=5.0, h_switch=0.5, r_mid=5.5, dsf_alpha=0.2, gamma=1.0,
                    temperature=300.0, eps0=0.1, eps_mode=1, skin=0.2, skin_outer=0.3)
# the same boxes under Ewald with the headline's settings (r_E 9 A fits the 18.6 A boxes)
ENSEMBLE_EW_JUMP = ENSEMBLE_DSF | EWALD | dict(r_cut=9.0, ring_r=[], lj_long_mode=2, skin=0.3, skin_outer=0.3,
                                               eps0=2.0)
ENSEMBLE_EW_BAOAB = ENSEMBLE_DSF | EWALD | dict(r_cut=9.0, skin=0.3, skin_outer=0.3)


def ensemble_leg(args, M, stream, device):
    """The batched ensemble, every replica advanced by the same launches:
    aggregate ns/day of JUMP and BAOAB (DSF, 1 fs), and under Ewald of
    JUMP-RESPA1 and BAOAB-RESPA1 (1:2:4 fs) with the mean temperature and the
    oxygen self-diffusion over all replicas, matched against BAOAB at 1 fs."""
    from paper_2412_15073_gb300 import systems
    sizes = systems.replica_sizes(64, seed=1)
    syss = [systems.water_box(n, seed=100 + k) for k, n in enumerate(sizes)]
    atoms = sum(s.n for s in syss)
    relax(M, None, ENSEMBLE_DSF, args.equil // 2, 77, device, stream, 64, syss)
    out = {"replicas": 64, "atoms": atoms, "sizes_atoms": [min(sizes) * 3, max(sizes) * 3]}

    def engine(seed, params, syss_=syss):
        e = M.Engine(precision=M.MD_MIXED, seed=seed, device=device, stream=stream.cuda_stream, max_replicas=64)
        for r, s in enumerate(syss_):
            e.set_system(r, s, **params)
        return e

    steps = 100
    dsf = {"params": "r_E 9 A, r_c 5 A, rings of r_mid 5.5 A, DSF 0.2/A, eps0 0.1, skin 0.2 A, 1 fs"}
    for name, seed, meth in (("jump", 78, "jump"), ("baoab", 79, "baoab")):
        e = engine(seed, ENSEMBLE_DSF)
        fn = getattr(e, meth)
        fn(args.warmup)
        t = timed(fn, steps, stream)
        Ts = [e.observables(r)["temperature"] for r in range(64)]
        dsf[name] = {"ns_per_day_aggregate": ns_per_day(64 * steps * DT_FS, t), "ms_per_step": t / steps * 1e3,
                     "T_mean": float(np.mean(Ts)), "T_min": float(np.min(Ts)), "T_max": float(np.max(Ts))}
        e.close()
    dsf["speed_ratio"] = dsf["jump"]["ns_per_day_aggregate"] / dsf["baoab"]["ns_per_day_aggregate"]
    dsf["steps"] = steps
    out["dsf"] = dsf
    # Ewald, matched: D and T averaged over the replicas (oxygens of all replicas)
    ew_syss = [s.copy() for s in syss]
    relax(M, None, ENSEMBLE_EW_BAOAB, args.equil // 2, 76, device, stream, 64, ew_syss)
    ew = {"params": "Ewald a 0.42/A real space to 9 A + smooth PME (order 6, 0.8 A grid per box), r_c 6 A, "
                    "JUMP-RESPA1 eps0 2 one ring, 1:2:4 fs vs BAOAB-RESPA1 1:2:4 fs; reference BAOAB 1 fs"}
    mass = np.concatenate([s.mass for s in ew_syss])
    for name, seed, meth, params in (("baoab_1fs", 81, "baoab", ENSEMBLE_EW_BAOAB),
                                     ("jump_respa1_D4", 82, "jump_respa1", ENSEMBLE_EW_JUMP),
                                     ("baoab_respa1_D4", 83, "baoab_respa1", ENSEMBLE_EW_BAOAB)):
        e = engine(seed, params, ew_syss)
        per = 1 if meth == "baoab" else 4
        run = (lambda k, e=e: e.baoab(k)) if meth == "baoab" else \
            (lambda k, e=e, m=meth: getattr(e, m)(k, 1.0, 2, 2))
        try:
            run(max(1, 120 // per))
            cyc = EW_WINDOW_FS // per
            t = timed(run, cyc, stream)
            r = {"ns_per_day_aggregate": ns_per_day(64 * cyc * per * DT_FS, t), "ms_per_fs": t / (cyc * per) * 1e3}
            ms, _ = profiled(e, run, 48 // per)
            r["class_ms_per_fs"] = {c: round(float(m) / 48, 4) for c, m in zip(CLASSES, ms)}
            if args.ens_dwindow > 0:
                r["D"], r["T_mean"] = ensemble_diffusion(e, lambda k: run(k // per), args.ens_dwindow, 24,
                                                         [s.box for s in ew_syss], mass)
            ew[name] = r
        except M.MDError as ex:
            ew[name] = {"error": str(ex)}
        e.close()
    ref = ew.get("baoab_1fs", {})
    for k in ("jump_respa1_D4", "baoab_respa1_D4"):
        if "ns_per_day_aggregate" in ew.get(k, {}):
            ew[k]["ns_per_day"] = ew[k]["ns_per_day_aggregate"]
            matched_flags(ew[k], ref)
    if "ns_per_day_aggregate" in ew.get("jump_respa1_D4", {}) and "ns_per_day_aggregate" in ew.get("baoab_respa1_D4", {}):
        ew["jump_over_baoab_respa1"] = ew["jump_respa1_D4"]["ns_per_day_aggregate"] / ew["baoab_respa1_D4"]["ns_per_day_aggregate"]
    ew["best_matched"] = best_matched({k: v for k, v in ew.items() if isinstance(v, dict) and k != "baoab_1fs"} |
                                      ({"baoab_1fs": ref | {"matched": True, "ns_per_day": ref["ns_per_day_aggregate"]}}
                                       if "ns_per_day_aggregate" in ref else {}))
    ew["D_window_ps"] = args.ens_dwindow * 1e-3
    out["ewald"] = ew
    return out


def ensemble_diffusion(e, integ, steps, every, boxes, mass):
    """D and mean T over all replicas of a batched engine (oxygens of every
    replica in one Einstein fit; 3N degrees of freedom over all atoms)"""
    R = len(boxes)
    xs, ts = [], []
    for k in range(steps // every + 1):
        X, V = [], []
        for r in range(R):
            x, v, img, _ = e.state(r)
            X.append((x + img * boxes[r])[::3])
            V.append(v)
        xs.append(np.concatenate(X))
        V = np.concatenate(V)
        ts.append((mass[:, None] * V * V).sum() / (3 * len(mass) * 0.0019872041 * 418.4))
        if k < steps // every:
            integ(every)
    X = np.stack(xs)
    nt = X.shape[0]
    lags = np.arange(1, nt)
    msd = np.array([((X[l:] - X[:-l]) ** 2).sum(-1).mean() for l in lags])
    t = lags * every * DT_FS * 1e-3
    sel = (lags >= 0.2 * (nt - 1)) & (lags <= 0.8 * (nt - 1))
    return np.polyfit(t[sel], msd[sel], 1)[0] / 6.0 * 10.0, float(np.mean(ts))


def million_leg(args, M, stream, device):
    """The heterogeneous 1,000,000-atom system (water around a dense sphere of
    50,002 charged LJ beads, 229 A box): under DSF (r_E 10, r_c 5 A; delta 1,
    kappa 2, Delta 2 fs, the largest stable outer step of BAOAB-RESPA1 there)
    and under Ewald with the headline's settings (1:2:4 fs) with D and T of
    the oxygens, matched against BAOAB at 1 fs."""
    from paper_2412_15073_gb300 import systems
    w = systems.water_with_beads(seed=2)
    relax(M, w, DSF | {"skin": 0.5}, 200, 91, device, stream)
    out = {"atoms": w.n, "box": w.box}

    def engine(seed, params):
        e = M.Engine(precision=M.MD_MIXED, seed=seed, device=device, stream=stream.cuda_stream)
        e.set_system(0, w, **params)
        return e

    dsf = {"levels": "delta 1 fs, kappa 2 fs, Delta 2 fs"}
    cyc = 20
    for name, seed, meth, params in (("jump_respa1", 92, "jump_respa1", DSF_JUMP),
                                     ("baoab_respa1", 93, "baoab_respa1", DSF | {"skin": 0.5})):
        e = engine(seed, params)
        run = lambda k, e=e, m=meth: getattr(e, m)(k, 1.0, 2, 1)
        run(3)
        c0 = e.observables()
        t = timed(run, cyc, stream)
        c1 = e.observables()
        dsf[name] = {"ns_per_day": ns_per_day(cyc * 2 * DT_FS, t), "ms_per_fs": t / (cyc * 2) * 1e3,
                     "T": c1["temperature"], "error_flags": c1["error_flags"]}
        if meth == "jump_respa1":
            dsf[name]["proposals_per_atom_fs"] = (c1["jump_proposals"] - c0["jump_proposals"]) / (w.n * cyc * 2)
        e.close()
    dsf["speed_ratio"] = dsf["jump_respa1"]["ns_per_day"] / dsf["baoab_respa1"]["ns_per_day"]
    out["dsf"] = dsf
    # Ewald: the full Coulomb sum of the bead sphere relaxes first at a short step and strong friction
    relax(M, w, EW_BAOAB, 200, 94, device, stream, gamma=50.0, dt_fs=0.5)
    relax(M, w, EW_BAOAB, 200, 98, device, stream)
    oxy_mass = w.mass
    ew = {}
    for name, seed, meth, params in (("baoab_1fs", 95, "baoab", EW_BAOAB),
                                     ("jump_respa1_D4", 96, "jump_respa1", EW_JUMP),
                                     ("baoab_respa1_D4", 97, "baoab_respa1", EW_BAOAB)):
        e = engine(seed, params)
        per = 1 if meth == "baoab" else 4
        run = (lambda k, e=e: e.baoab(k)) if meth == "baoab" else \
            (lambda k, e=e, m=meth: getattr(e, m)(k, 1.0, 2, 2))
        try:
            run(max(1, 24 // per))
            cyc = 96 // per
            t = timed(run, cyc, stream)
            r = {"ns_per_day": ns_per_day(cyc * per * DT_FS, t), "ms_per_fs": t / (cyc * per) * 1e3}
            ms, _ = profiled(e, run, 24 // per)
            r["class_ms_per_fs"] = {c: round(float(m) / 24, 4) for c, m in zip(CLASSES, ms)}
            if args.mil_dwindow > 0:
                r["D"], r["T_mean"] = diffusion(e, lambda k: run(k // per), args.mil_dwindow, 24, w.box, DT_FS,
                                                oxy_mass)
            ew[name] = r
        except M.MDError as ex:
            ew[name] = {"error": str(ex)}
        e.close()
    ref = ew.get("baoab_1fs", {})
    for k in ("jump_respa1_D4", "baoab_respa1_D4"):
        if "ns_per_day" in ew.get(k, {}):
            matched_flags(ew[k], ref)
    if "ns_per_day" in ew.get("jump_respa1_D4", {}) and "ns_per_day" in ew.get("baoab_respa1_D4", {}):
        ew["jump_over_baoab_respa1"] = ew["jump_respa1_D4"]["ns_per_day"] / ew["baoab_respa1_D4"]["ns_per_day"]
    ew["best_matched"] = best_matched(ew | ({"baoab_1fs": ref | {"matched": True}} if "ns_per_day" in ref else {}))
    ew["D_window_ps"] = args.mil_dwindow * 1e-3
    ew["note"] = "D of the water oxygens and of the beads' first atom stride (atoms 0, 3, 6, ...)"
    out["ewald"] = ew
    return out


CM1_PER_INV_FS = 1e15 / 2.99792458e10      # 1/fs in cm^-1


def spectra_leg(args, M, engine):
    """Velocity spectra (mass-weighted VACF, Hann-windowed cosine transform) of
    BAOAB (1 fs) and of BAOAB-RESPA1 and JUMP-RESPA1 (1:2:6 fs) under Ewald
    electrostatics, recorded after every 1 fs step (Sec. 4: resonance peaks of
    the multiple-time-step integrators): the share of the weight above
    4200 cm^-1, where only integrator artefacts live, and the strongest
    artefact peak."""
    T, K = args.spectra, min(2048, args.spectra // 2)
    out = {"samples": T, "lags": K, "bin_cm1": CM1_PER_INV_FS / (2 * K * DT_FS), "window": "Hann",
           "electrostatics": "Ewald as in the headline"}
    # the paper's BAOAB setting moves more of the Coulomb sum into the
    # reciprocal part (a = 0.5446/A, 120^3 grid) than its JUMP setting (a = 0.42/A)
    paper_baoab = {"dsf_alpha": 0.5446, "pme_spacing": BOX / 120}
    runs = [("baoab_1fs", 7, "baoab", 1, EW_BAOAB),
            ("baoab_respa1_D6_a0.5446", 8, "baoab_respa1", 3, EW_BAOAB | paper_baoab),
            ("baoab_respa1_D6_a0.42", 8, "baoab_respa1", 3, EW_BAOAB),
            ("jump_respa1_D6_a0.42", 9, "jump_respa1", 3, EW_JUMP | {"eps0": 0.1})]
    for name, seed, meth, q, params in runs:
        e = engine(seed, params)
        per = 1 if meth == "baoab" else 2 * q
        run = (lambda k: e.baoab(k)) if meth == "baoab" else (lambda k, e=e, m=meth, q=q: getattr(e, m)(k // (2 * q), 1.0, 2, q))
        try:
            run(120 // per * per)
            e.vacf_start(T)
            run(-(-T // per) * per)
            C, S, n = e.vacf(K)
            nu = np.arange(K) * CM1_PER_INV_FS / (2 * K * DT_FS)
            Sp = np.clip(S, 0, None)
            hi = nu > 4200
            st = (nu > 3000) & (nu < 4200)
            out[name] = {"samples": n, "T": e.observables()["temperature"],
                         "share_above_4200": float(Sp[hi].sum() / Sp.sum()),
                         "stretch_peak_cm1": float(nu[st][np.argmax(Sp[st])]),
                         "top_artefact_cm1": float(nu[hi][np.argmax(Sp[hi])]),
                         "top_artefact_rel": float(Sp[hi].max() / Sp[st].max())}
            e.vacf_start(0)
        except M.MDError as ex:
            out[name] = {"error": str(ex)}
        e.close()
    return out


def skin_sweep(args, M, engine, stream):
    """List skins of the headline runs: JUMP-RESPA1 and BAOAB-RESPA1 (1:2:4 fs,
    Ewald) timed over EW_WINDOW_FS for each inner skin and each width of the
    outer candidate shell beyond it (the headline settings: 0.4 A and 1.1 A)"""
    out = {"window_fs": EW_WINDOW_FS}
    for name, seed, meth, params in (("jump_respa1", 5, "jump_respa1", EW_JUMP),
                                     ("baoab_respa1", 6, "baoab_respa1", EW_BAOAB)):
        res = {}
        for skin, extra in [(sk, ex) for sk in args.sweep_skin for ex in args.sweep_outer]:
            e = engine(seed, params | {"skin": skin, "skin_outer": skin + extra})
            run = lambda k, e=e, m=meth: getattr(e, m)(k, 1.0, M_MID, N_OUT)
            try:
                run(30)
                cyc = EW_WINDOW_FS // CYCLE_FS
                c0 = e.observables()
                t = timed(run, int(cyc), stream)
                c1 = e.observables()
                res[f"{skin:g}+{extra:g}"] = {"ns_per_day": ns_per_day(cyc * CYCLE_FS, t),
                                    "rebuilds_per_ps": (c1["list_rebuilds"] - c0["list_rebuilds"]) / (cyc * CYCLE_FS * 1e-3),
                                    "outer_rebuilds_per_ps": (c1["outer_rebuilds"] - c0["outer_rebuilds"]) /
                                                             (cyc * CYCLE_FS * 1e-3)}
            except M.MDError as ex:
                res[f"{skin:g}+{extra:g}"] = {"error": str(ex)}
            e.close()
        out[name] = res
    return out


def list_entry_counts(e, n_atoms, kinds=(0, 4), sample=400, seed=3):
    """mean jump-list lengths (ring 0, LJ) over sampled atoms"""
    rng = np.random.default_rng(seed)
    at = rng.choice(n_atoms, min(sample, n_atoms), replace=False)
    return {k: float(np.mean([len(e.get_list(k, int(i))) for i in at])) for k in kinds}


def inner_list_roofline(ms_total, groups, rebuilds, w, x, e, hbm, peak_kind):
    """HBM roofline of the inner list filter of the headline JUMP-RESPA1
    run: a rebuild streams every atom's outer candidates and stores the kept
    entries of its short, ring and LJ lists (algorithmic bytes: see the
    INNER_BYTES constants); achieved = those bytes times the rebuilds over the
    device time of all the kernel's launches (the launches that found no list
    to rebuild cost a flag read per atom and are included)."""
    from scipy.spatial import cKDTree
    n = w.n
    t = cKDTree(np.mod(x, BOX), boxsize=BOX)
    def per_atom(r):
        return 2.0 * len(t.query_pairs(r, output_type="ndarray")) / n
    p = EW_JUMP
    n_outer = per_atom(p["r_cut"] + p["skin_outer"])
    n_short = per_atom(p["r_split"] + p["skin"])
    lists = list_entry_counts(e, n)
    n_inner = n_short + lists[0] + lists[4]
    per_rebuild_s = ms_total / max(rebuilds, 1) * 1e-3
    nbytes = n * (INNER_BYTES_PER_CAND * n_outer + INNER_BYTES_PER_ENTRY * n_inner + INNER_BYTES_PER_ATOM)
    achieved = nbytes / per_rebuild_s / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": None,
            "traffic_earlier": {"bytes": INNER_TRAFFIC_NCU_EARLIER,
                                "note": "ncu, one rebuild launch of k_inner_lists<69> (one-ring JUMP lists) on this "
                                        "workload, taken before the kernel's exit for idle launches was added"},
            "kernel": "k_inner_lists (inner list filter of the list rebuild)",
            "bytes_per_launch": nbytes, "outer_candidates_per_atom": n_outer, "inner_entries_per_atom": n_inner,
            "ms_per_launch": per_rebuild_s * 1e3, "launches": int(groups), "rebuilds": int(rebuilds),
            "ms_all_launches": ms_total, "peak_kind": peak_kind,
            "bytes_model": f"{INNER_BYTES_PER_CAND} B per outer candidate + {INNER_BYTES_PER_ENTRY} B per kept "
                           f"entry + {INNER_BYTES_PER_ATOM} B per atom"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20, help="timed headline steps (4 fs cycles)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=32, help="atoms of the single-thread CPU sample")
    ap.add_argument("--equil", type=int, default=1000,
                    help="BAOAB steps at gamma = 20/ps from the lattice start before timing (0 = none)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--dwindow", type=int, default=40000, help="fs of each 96,000-atom run for D (0 = skip)")
    ap.add_argument("--psteps", type=int, default=10000, help="steps of each run of the precision leg")
    ap.add_argument("--ens-dwindow", type=int, default=6000, help="fs of each ensemble run for D (0 = skip)")
    ap.add_argument("--mil-dwindow", type=int, default=2400, help="fs of each 10^6-atom run for D (0 = skip)")
    ap.add_argument("--only", default="all",
                    choices=["all", "headline", "ewald", "dsf", "dsf_sweep", "skin_sweep", "spectra", "ensemble", "million",
                             "precision",
                             "jump", "baoab", "jump_respa1_ewald", "baoab_respa1_ewald"])
    ap.add_argument("--ensemble", type=int, default=1, help="also time the batched 64-replica ensemble")
    ap.add_argument("--million", type=int, default=1, help="also time the 1,000,000-atom heterogeneous system")
    ap.add_argument("--spectra", type=int, default=0, help="1 fs samples of the velocity-spectra leg (0 = skip)")
    ap.add_argument("--ewald-runs", nargs="*", default=None, help="only these Ewald runs (plus the 1 fs reference)")
    ap.add_argument("--sweep-rc", type=float, nargs="*", default=[5.0, 6.0, 7.0])
    ap.add_argument("--sweep-eps0", type=float, nargs="*", default=[0.1, 1.0, 2.0])
    ap.add_argument("--sweep-skin", type=float, nargs="*", default=[0.3, 0.4, 0.5, 0.6, 0.8])
    ap.add_argument("--sweep-outer", type=float, nargs="*", default=[1.1])
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import paper_2412_15073_gb300 as M
    from paper_2412_15073_gb300 import systems

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    ranks = Ranks("nccl")
    world, rank, local = ranks.world, ranks.rank, ranks.local
    barrier, max_over_ranks = ranks.barrier, ranks.max
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    pk, peak_kind = peaks()
    stream = torch.cuda.current_stream()

    if args.only == "ensemble":
        out = ensemble_leg(args, M, stream, local)
        if rank == 0:
            print(json.dumps({"ensemble": out}), flush=True)
        ranks.close()
        return
    if args.only == "precision":
        out = precision_leg(args, M, stream, local)
        if rank == 0:
            print(json.dumps({"precision": out}), flush=True)
        ranks.close()
        return
    if args.only == "million":
        t0 = time.perf_counter()
        out = million_leg(args, M, stream, local)
        out["wall_s"] = time.perf_counter() - t0
        if rank == 0:
            print(json.dumps({"million": out}), flush=True)
        ranks.close()
        return

    w = systems.water_box(N_MOL, box=BOX, seed=0)
    n = w.n
    if args.equil > 0:
        # relax the lattice start at strong friction so every run starts at 300 K
        relax(M, w, DSF, args.equil, ranks.seed(99), local, stream)
    w_dsf = w.copy()
    w_ew = w.copy()
    if args.equil > 0 and args.only not in ("dsf", "dsf_sweep", "jump", "baoab"):
        relax(M, w_ew, EW_BAOAB, args.equil, ranks.seed(98), local, stream)

    def engine_on(sys_):
        def engine(seed, params):
            e = M.Engine(precision=M.MD_MIXED, seed=ranks.seed(seed), device=local, stream=stream.cuda_stream)
            e.set_system(0, sys_, **params)
            return e
        return engine

    eng_ew, eng_dsf = engine_on(w_ew), engine_on(w_dsf)

    if args.only in ("jump", "baoab", "jump_respa1_ewald", "baoab_respa1_ewald"):
        # profiling run: one integrator, no side measurements
        if args.only == "jump":
            e = eng_dsf(1, DSF_JUMP)
            fn = e.jump
        elif args.only == "baoab":
            e = eng_dsf(1, DSF_BAOAB)
            fn = e.baoab
        elif args.only == "jump_respa1_ewald":
            e = eng_ew(1, EW_JUMP)
            fn = lambda k: e.jump_respa1(k, 1.0, M_MID, N_OUT)
        else:
            e = eng_ew(1, EW_BAOAB)
            fn = lambda k: e.baoab_respa1(k, 1.0, M_MID, N_OUT)
        fn(args.warmup)
        torch.cuda.nvtx.range_push("timed")        # ncu --nvtx --nvtx-include timed/ selects these launches
        t = timed(fn, args.steps, stream)
        torch.cuda.nvtx.range_pop()
        fs = args.steps * (DT_FS if args.only in ("jump", "baoab") else CYCLE_FS)
        if rank == 0:
            print(json.dumps({"only": args.only, "ns_per_day": ns_per_day(fs, t), "ms_per_step": t / args.steps * 1e3,
                              "profile_launches": e.profile()[2].tolist()}))
        e.close()
        ranks.close()
        return
    if args.only == "ewald":
        out = ewald_runs(args, M, eng_ew, stream, world, max_over_ranks, barrier, w.mass, names=args.ewald_runs)
        if rank == 0:
            print(json.dumps({"ewald": out}), flush=True)
        ranks.close()
        return
    if args.only == "spectra":
        args.spectra = args.spectra or 4096
        out = spectra_leg(args, M, eng_ew)
        if rank == 0:
            print(json.dumps({"spectra": out}), flush=True)
        ranks.close()
        return
    if args.only == "skin_sweep":
        out = skin_sweep(args, M, eng_ew, stream)
        if rank == 0:
            print(json.dumps({"skin_sweep": out}), flush=True)
        ranks.close()
        return
    if args.only == "dsf_sweep":
        out = dsf_sweep(args, M, eng_dsf, stream, w.mass)
        if rank == 0:
            print(json.dumps({"dsf_sweep": out}), flush=True)
        ranks.close()
        return
    if args.only == "dsf":
        out = dsf_leg(args, M, eng_dsf, stream, world, max_over_ranks, barrier, w.mass, sms,
                      pk.get("sm_max_mhz", 2070.0), pk["hbm_gbs"], peak_kind)
        if rank == 0:
            print(json.dumps({"dsf": out}), flush=True)
        ranks.close()
        return

    # ---- headline: JUMP-RESPA1 vs BAOAB-RESPA1, K cycles each
    ej = eng_ew(1, EW_JUMP)
    eb = eng_ew(2, EW_BAOAB)
    run_j = lambda k: ej.jump_respa1(k, 1.0, M_MID, N_OUT)
    run_b = lambda k: eb.baoab_respa1(k, 1.0, M_MID, N_OUT)
    run_j(args.warmup)          # warm-up: autotuners, then the CUDA graph of a cycle is captured
    run_b(args.warmup)
    c0 = ej.observables()
    l0 = ej.profile()[2].sum()
    barrier()
    with Clocks(local) as clk:
        t_jump = timed(run_j, args.steps, stream)
        barrier()
        t_baoab = timed(run_b, args.steps, stream)
        barrier()
    launches = int(ej.profile()[2].sum() - l0)
    t_jump, t_baoab = max_over_ranks(t_jump), max_over_ranks(t_baoab)
    c1 = ej.observables()
    ob_b = eb.observables()
    clocks = clk.summary()
    clock_mhz = clocks["sm_mhz"] or pk.get("sm_max_mhz", 2070.0)
    fs = args.steps * CYCLE_FS
    jump_nsday = ns_per_day(world * fs, t_jump)
    baoab_nsday = ns_per_day(world * fs, t_baoab)
    # pair evaluations per cycle: short pairs per kappa step (2), the long
    # real-space pairs of BAOAB-RESPA1 per Delta; jump proposals of JUMP-RESPA1
    x_j, x_b = ej.state()[0], eb.state()[0]
    pairs_short = pair_counts(x_j, BOX, EW_JUMP["r_split"])
    pairs_full_b = pair_counts(x_b, BOX, EW_BAOAB["r_cut"])
    pairs_short_b = pair_counts(x_b, BOX, EW_BAOAB["r_split"])
    props = (c1["jump_proposals"] - c0["jump_proposals"]) / args.steps
    gpe = {"jump_respa1": world * (N_OUT * pairs_short + props) * args.steps / t_jump / 1e9,
           "baoab_respa1": world * (N_OUT * pairs_short_b + pairs_full_b) * args.steps / t_baoab / 1e9}
    # per-class device time of the headline JUMP-RESPA1 cycle (profiled run, plain launches)
    r0 = ej.observables()["list_rebuilds"]
    ms, groups = profiled(ej, run_j, 60)
    rebuilds = ej.observables()["list_rebuilds"] - r0
    top = int(np.argmax(ms))
    hbm = pk["hbm_gbs"]
    if CLASSES[top] == "list_inner":
        roof = inner_list_roofline(float(ms[top]), int(groups[top]), rebuilds, w_ew, x_j, ej, hbm, peak_kind)
    elif CLASSES[top] == "pair_force":
        roof = pair_roofline(float(ms[top]), int(groups[top]), pairs_short, sms, clock_mhz)
        roof["kernel"] = "k_force (short pairs of JUMP-RESPA1, and its slow-level LJ part)"
    elif CLASSES[top] == "velocity_phase":
        roof = cphase_roofline(float(ms[top]), int(groups[top]), props * 60, n, hbm, sms, clock_mhz, peak_kind)
    else:
        roof = {"bound": "hbm", "kernel_class": CLASSES[top], "achieved": None, "peak": hbm, "unit": "GB/s",
                "frac": None, "traffic": None, "note": "no byte model for this class"}
    roof["share_of_cycle"] = float(ms[top] / ms.sum())
    roof["class_ms_per_cycle"] = {c: round(float(m) / 60, 4) for c, m in zip(CLASSES, ms)}
    msb, _ = profiled(eb, run_b, 60)
    baoab_classes = {c: round(float(m) / 60, 4) for c, m in zip(CLASSES, msb)}
    e2e = None
    if not args.no_e2e:
        e2e = e2e_run(ej, run_j, args, M, torch, n, world, max_over_ranks, barrier, CYCLE_FS)
    ej.close()
    eb.close()
    if args.only == "headline":
        if rank == 0:
            print(json.dumps({"only": "headline", "value": jump_nsday, "baoab_respa1_ns_per_day": baoab_nsday,
                              "speedup_vs_baoab_respa1": jump_nsday / baoab_nsday, "ms_per_step": t_jump / args.steps * 1e3,
                              "gpu_launches": launches, "roofline": roof, "baoab_respa1_class_ms_per_cycle": baoab_classes,
                              "gpair_evals_per_s": gpe, "e2e": e2e, "clocks": clocks}), flush=True)
        ranks.close()
        return

    # ---- matched T and D (fixed windows, the same equilibrated start)
    ewald = ewald_runs(args, M, eng_ew, stream, world, max_over_ranks, barrier, w.mass, names=args.ewald_runs)
    bm = ewald["best_matched"]
    head = ewald.get("jump_respa1_D4", {})
    matched = {"workload": WORKLOAD, "criterion": ewald["criterion"], "reference": "BAOAB 1 fs",
               "D_window_ps": ewald["D_window_ps"], "headline_jump_run": "jump_respa1_D4",
               "headline_jump_matched": head.get("matched"), "headline_baoab_run": "baoab_respa1_D4",
               "headline_baoab_matched": ewald.get("baoab_respa1_D4", {}).get("matched"),
               "fastest_matched_jump": bm.get("jump"), "fastest_matched_baoab": bm.get("baoab"),
               "jump_over_baoab": bm.get("jump_over_baoab")}
    # without a matched BAOAB-RESPA1 run, the fastest matched BAOAB is the reference itself
    ref_ns = ewald.get("baoab_1fs", {}).get("ns_per_day")
    if "jump" in bm and "baoab" not in bm and ref_ns:
        matched["jump_over_reference_baoab_1fs"] = bm["jump"]["ns_per_day"] / ref_ns
    for k in ("jump_respa1_D4", "baoab_respa1_D4"):
        if ewald.get(k, {}).get("D_ratio_se") is not None:
            matched[k + "_D_ratio"] = [ewald[k]["D_ratio"], ewald[k]["D_ratio_se"]]

    # ---- DSF water (damped shifted force Coulomb): 1 fs JUMP vs BAOAB, rooflines
    dsf = dsf_leg(args, M, eng_dsf, stream, world, max_over_ranks, barrier, w.mass, sms, clock_mhz, hbm,
                  peak_kind)
    dsf["respa1"] = dsf_respa1(args, M, eng_dsf, stream, world, max_over_ranks, barrier)
    spectra = spectra_leg(args, M, eng_ew) if args.spectra > 0 else None
    ensemble = ensemble_leg(args, M, stream, local) if args.ensemble else None
    million = million_leg(args, M, stream, local) if args.million else None

    out = {"metric": METRIC, "value": jump_nsday, "unit": "ns/day", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_jump / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+i64+f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "atoms": n, "fs_per_step": CYCLE_FS, "global_batch": world,
                      "parallelism": "replicas",
                      "l2": "working set (neighbour lists ~0.4 GB, PME grids) above the 129 MB L2; consecutive "
                            "cycles, no flush"},
           "jump_respa1_ns_per_day": jump_nsday, "baoab_respa1_ns_per_day": baoab_nsday,
           "speedup_vs_baoab_respa1": jump_nsday / baoab_nsday,
           "gpair_evals_per_s": gpe,
           "T_end": {"jump_respa1": c1["temperature"], "baoab_respa1": ob_b["temperature"]},
           "jump_stats": {"proposals_per_atom_cycle": props / n,
                          "accept_frac": (c1["jump_accepts"] - c0["jump_accepts"]) /
                                         max(c1["jump_proposals"] - c0["jump_proposals"], 1),
                          "list_rebuilds": c1["list_rebuilds"] - c0["list_rebuilds"]},
           "matched": matched,
           "ewald": ewald,
           "dsf": dsf,
           "roofline": roof,
           "roofline_cphase": dsf["roofline_cphase"],
           "pair_roofline": dsf["pair_roofline"],
           "baoab_respa1_class_ms_per_cycle": baoab_classes,
           "spectra": spectra, "ensemble": ensemble, "million": million,
           "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
           "device": {"sms": sms, "peaks": peak_kind}}
    parts = [f"fastest matched JUMP {bm['jump']['run']} {bm['jump']['ns_per_day']:.1f} ns/day" if "jump" in bm
             else "no JUMP run matched"]
    if "baoab" in bm:
        parts.append(f"fastest matched BAOAB {bm['baoab']['run']} {bm['baoab']['ns_per_day']:.1f} ns/day")
    elif ref_ns:
        parts.append(f"no BAOAB-RESPA1 run matched; reference BAOAB 1 fs {ref_ns:.1f} ns/day")
    if "jump_over_baoab" in bm:
        parts.append(f"ratio {bm['jump_over_baoab']:.3f}")
    elif "jump_over_reference_baoab_1fs" in matched:
        parts.append(f"ratio to the reference {matched['jump_over_reference_baoab_1fs']:.3f}")
    summ = {"ewald_96k": "; ".join(parts)}
    if "jump" in dsf:
        summ["dsf_96k"] = (f"JUMP {dsf['jump_ns_per_day']:.1f} vs BAOAB {dsf['baoab_ns_per_day']:.1f} ns/day at 1 fs; "
                           f"D ratio {dsf['jump'].get('D_ratio', float('nan')):.3f}, T ratio "
                           f"{dsf['jump'].get('T_ratio', float('nan')):.4f}: "
                           f"{'matched' if dsf['jump'].get('matched') else 'not matched'}")
    out["matched_summary"] = summ
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        n_all = args.cpu_sample * oracle.get_threads()
        ((t_one, thr1, _), (t_all, thr, _)), tg = headline_oracle_cost(w_ew, [(args.cpu_sample, 1, 1), (n_all, 1, 0)])
        sample = (f"{{n}} of 96,000 atoms, each with its per-atom work of one JUMP-RESPA1 cycle (three O(N) "
                  f"nonbonded passes, four C' phases), plus the whole-system parts timed once (four bonded "
                  f"gradients, one smooth-PME sum: {tg:.1f} s); list builds excluded; scaled to the full cycle")
        out["cpu_baseline"] = {"value": ns_per_day(CYCLE_FS, t_all), "unit": "ns/day", "cores": thr, "kind": "oracle",
                               "sample": sample.format(n=n_all),
                               "single_thread": {"value": ns_per_day(CYCLE_FS, t_one), "unit": "ns/day",
                                                 "cores": thr1, "sample": sample.format(n=args.cpu_sample)}}
    if rank == 0:
        print(json.dumps(out), flush=True)
    ranks.close()


if __name__ == "__main__":
    main()
