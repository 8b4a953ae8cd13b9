"""Writes oracle_648_ewald.json: what the FP64 oracle computes for the
648-atom water (216 flexible waters, 18.643 A box, lattice start from seed 0)
under Ewald electrostatics (erfc(a r)/r to 9 A with a = 0.42/A, smooth PME of
order 6 on a 0.8 A grid, split at 6 A, one ring, the LJ long part at the slow
level) after 60 innermost steps of JUMP-RESPA1 and of BAOAB-RESPA1 (1:2:6 fs).
It calls the oracle only; the file is a regression record of the oracle,
checked by tests/test_oracle_golden.py.

    python tests/golden/make_golden_ewald.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "..", ".."))

import oracle  # noqa: E402
from paper_2412_15073_gb300 import systems  # noqa: E402

PARAMS = dict(r_cut=9.0, r_split=6.0, h_switch=0.5, dsf_alpha=0.42, gamma=1.0, temperature=300.0,
              eps0=2.0, eps_mode=1, skin=0.2, skin_outer=0.3, ring_r=[], lj_long_mode=2,
              coulomb_mode=1, pme_order=6, pme_spacing=0.8)
OUTER = 10


def run(integrator):
    w = systems.water_box(216, box=18.643, seed=0)
    o = oracle.Oracle(w, seed=0, replica=0, **PARAMS)
    rc = getattr(o, integrator)(OUTER, 1.0, 2, 3)
    x, v, img, _ = o.state()
    e = o.energy()
    return {"rc": int(rc), "step": int(o.step), "counters": [int(c) for c in o.counters()],
            "energy": [float(z) for z in e], "x_first": x[:4].tolist(), "v_first": v[:4].tolist(),
            "x_sum": float(x.sum()), "v_sq_sum": float((v * v).sum())}


if __name__ == "__main__":
    oracle.build()
    import platform
    out = {"workload": "216 waters, 18.643 A, seed 0; " + json.dumps(PARAMS) + f"; {OUTER} outer steps of 6 fs",
           "machine": platform.machine(), "jump_respa1": run("jump_respa1"), "baoab_respa1": run("baoab_respa1")}
    with open(os.path.join(HERE, "oracle_648_ewald.json"), "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", os.path.join(HERE, "oracle_648_ewald.json"))
