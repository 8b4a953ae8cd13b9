"""The oracle against its own record (tests/golden/oracle_648_1000.json,
written by tests/golden/make_golden.py, which calls the oracle only) on the
plain 648-atom workload: 1000 steps of BAOAB and of JUMP in FP64. A change to
the oracle's arithmetic shows up here. On the machine type that wrote the
record the state repeats it exactly; elsewhere (another libm) to 1e-6.""" 
import json
import os
import platform

import numpy as np
import pytest

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.mark.parametrize("integrator", ["baoab", "jump"])
def test_oracle_repeats_its_record(oracle_mod, integrator):
    import sys
    sys.path.insert(0, HERE)
    import make_golden
    rec = json.load(open(os.path.join(HERE, "oracle_648_1000.json")))
    got = make_golden.run(integrator)
    ref = rec[integrator]
    assert got["rc"] == ref["rc"] == 0 and got["step"] == ref["step"] == 1000
    if platform.machine() == rec["machine"]:
        # the state repeats bit for bit; the energy sums are threaded (order of
        # the partial sums varies), so they repeat to rounding
        np.testing.assert_allclose(got.pop("energy"), ref["energy"], rtol=1e-12)
        assert got == {k: v for k, v in ref.items() if k != "energy"}
    else:
        np.testing.assert_allclose(got["energy"], ref["energy"], rtol=1e-6)
        np.testing.assert_allclose(got["x_first"], ref["x_first"], atol=1e-6)


@pytest.mark.parametrize("integrator", ["jump_respa1", "baoab_respa1"])
def test_oracle_repeats_its_ewald_record(oracle_mod, integrator):
    """the same for the Ewald / smooth-PME path (tests/golden/oracle_648_ewald.json,
    written by tests/golden/make_golden_ewald.py): 60 innermost steps of the
    RESPA1 pair at the paper's settings"""
    import sys
    sys.path.insert(0, HERE)
    import make_golden_ewald
    rec = json.load(open(os.path.join(HERE, "oracle_648_ewald.json")))
    got = make_golden_ewald.run(integrator)
    ref = rec[integrator]
    assert got["rc"] == ref["rc"] == 0 and got["step"] == ref["step"] == 60
    if platform.machine() == rec["machine"]:
        np.testing.assert_allclose(got.pop("energy"), ref["energy"], rtol=1e-12)
        assert got == {k: v for k, v in ref.items() if k != "energy"}
    else:
        np.testing.assert_allclose(got["energy"], ref["energy"], rtol=1e-6)
        np.testing.assert_allclose(got["x_first"], ref["x_first"], atol=1e-6)
