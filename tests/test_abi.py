"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point include/md.h declares (no compute calls: this runs on the CPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "md.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(md_[a-z_0-9]+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2412_15073_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = header_functions()
    for n in ("md_init", "md_set_system", "md_step_baoab", "md_step_jump", "md_step_jump_respa",
              "md_step_jump_respa1", "md_observables", "md_finalize"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    import ctypes
    lib = ctypes.CDLL(libpath)
    for n in header_functions():
        assert hasattr(lib, n), n


def test_binding_lists_the_header(libpath):
    import paper_2412_15073_gb300 as M
    assert sorted(M.SYMBOLS) == header_functions()
    L = M.load_library(libpath)
    assert L.md_last_error(None).decode()


def test_init_rejects_bad_config_without_gpu(libpath):
    """Argument checks happen before any device call."""
    import ctypes
    import paper_2412_15073_gb300 as M
    L = M.load_library(libpath)
    h = ctypes.c_void_p()
    cfg = M.MdConfig(7, 0, 0, None, 1, 0, 0)
    assert L.md_init(ctypes.byref(h), ctypes.byref(cfg)) == -1
    assert b"precision" in L.md_last_error(None)
    cfg = M.MdConfig(1, 0, 0, None, 0, 0, 0)
    assert L.md_init(ctypes.byref(h), ctypes.byref(cfg)) == -1
    cfg = M.MdConfig(1, 0, 0, None, 1, 0, 3)
    assert L.md_init(ctypes.byref(h), ctypes.byref(cfg)) == -1


def test_no_cpu_fallback_in_the_product_path():
    """The package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2412_15073_gb300")
    for dp, _, fs in os.walk(pkg):
        for f in fs:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dp, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "liboracle" not in txt, f


class _StubLib:
    """stands in for libmdjump.so: records the md_system the binding builds"""

    def __init__(self):
        self.sys = None

    def md_set_system(self, h, replica, ref):
        s = ref._obj
        self.sys = {k: getattr(s, k) for k, _ in s._fields_}
        self.sys["ring_r"] = list(s.ring_r)
        return 0

    def md_set_state(self, *args):
        return 0


def _stub_engine():
    import paper_2412_15073_gb300 as M
    e = M.Engine.__new__(M.Engine)
    e.L, e.h, e.n = _StubLib(), None, {}
    return e


def test_binding_marshals_the_system_and_checks_sizes():
    """argument marshalling of set_system / set_state on the host (no GPU):
    counts, ring edges and electrostatics reach md_system; arrays whose sizes
    disagree with n_atoms are refused before the library reads them"""
    from paper_2412_15073_gb300 import systems
    w = systems.water_box(8, box=12.0, seed=0)
    e = _stub_engine()
    e.set_system(0, w, ring_r=[6.0, 7.5], coulomb_mode=1, pme_order=8, lj_long_mode=2, skin=0.25)
    s = e.L.sys
    assert s["n_atoms"] == w.n == 24 and s["n_bonds"] == len(w.bond_k) and s["n_angles"] == len(w.angle_k)
    assert s["n_excl"] == w.excl.shape[0] and s["n_types"] == w.lj_eps.shape[0]
    assert s["n_rings"] == 3 and s["ring_r"][:2] == [6.0, 7.5]
    assert (s["coulomb_mode"], s["pme_order"], s["lj_long_mode"]) == (1, 8, 2)
    assert s["skin"] == 0.25 and s["skin_outer"] == 0.25
    with pytest.raises(ValueError):
        e.set_system(0, w, ring_r=[5.5, 6.0, 7.0, 8.0])
    bad = w.copy()
    bad.v = bad.v[:-1]
    with pytest.raises(ValueError, match="v has"):
        e.set_system(0, bad)
    bad = w.copy()
    bad.charge = bad.charge[:-2]
    with pytest.raises(ValueError, match="charge has"):
        e.set_system(0, bad)
    e.set_state(0, w.x, w.v)
    with pytest.raises(ValueError, match="v has"):
        e.set_state(0, w.x, w.v[:3])


def test_noalloc_rejects_oversized_inputs_before_any_device_call(libpath):
    """md_nb_gradient_noalloc checks its scratch limits on the host: too many
    atoms, or a box / r_cut ratio that needs more cells than the static
    array holds, is refused with MD_EINVAL before any pointer is read."""
    import numpy as np
    import paper_2412_15073_gb300 as M
    L = M.load_library(libpath)
    one = np.zeros(8)
    p = M._ptr(one)
    # 200,000 atoms: above MD_NOALLOC_MAX_ATOMS
    assert L.md_nb_gradient_noalloc(p, p, p, None, 200_000, 1000.0, 1, p, p, 9.0, 5.0, 0.5, 0.2, 0, p, None) == -1
    assert b"MD_NOALLOC_MAX_ATOMS" in L.md_last_error(None)
    # 10 atoms in a 330 A box at r_cut 9 A: 36^3 = 46,656 cells, above MD_NOALLOC_MAX_CELLS
    assert L.md_nb_gradient_noalloc(p, p, p, None, 10, 330.0, 1, p, p, 9.0, 5.0, 0.5, 0.2, 0, p, None) == -1
    assert b"MD_NOALLOC_MAX_CELLS" in L.md_last_error(None)
    # an unknown weight is refused as well
    assert L.md_nb_gradient_noalloc(p, p, p, None, 10, 100.0, 1, p, p, 9.0, 5.0, 0.5, 0.2, 3, p, None) == -1
    assert b"weight" in L.md_last_error(None)
