"""Writes oracle_648_1000.json: what the FP64 oracle computes for the plain
648-atom workload (216 flexible waters, 18.643 A box, lattice start from seed
0, DSF alpha 0.2 with a 9 A cutoff, split at 5 A, 300 K, gamma 1/ps, 1 fs)
after 1000 steps of BAOAB and of JUMP. It calls the oracle only; the file is
a regression record of the oracle, checked by tests/test_oracle_golden.py.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "..", ".."))

import oracle  # noqa: E402
from paper_2412_15073_gb300 import systems  # noqa: E402

PARAMS = dict(r_cut=9.0, r_split=5.0, h_switch=0.5, r_mid=5.5, dsf_alpha=0.2, gamma=1.0,
              temperature=300.0, eps0=0.1, eps_mode=1, skin=0.2, skin_outer=0.3)
STEPS = 1000


def run(integrator):
    w = systems.water_box(216, box=18.643, seed=0)
    o = oracle.Oracle(w, seed=0, replica=0, **PARAMS)
    rc = getattr(o, integrator)(STEPS)
    x, v, img, _ = o.state()
    e = o.energy()
    return {"rc": int(rc), "step": int(o.step), "counters": [int(c) for c in o.counters()],
            "energy": [float(z) for z in e], "x_first": x[:4].tolist(), "v_first": v[:4].tolist(),
            "x_sum": float(x.sum()), "v_sq_sum": float((v * v).sum())}


if __name__ == "__main__":
    oracle.build()
    import platform
    out = {"workload": "216 waters, 18.643 A, seed 0; " + json.dumps(PARAMS) + f"; {STEPS} steps of 1 fs",
           "machine": platform.machine(), "baoab": run("baoab"), "jump": run("jump")}
    with open(os.path.join(HERE, "oracle_648_1000.json"), "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", os.path.join(HERE, "oracle_648_1000.json"))
