"""GB300 (sm_103a) Velocity Jumps molecular dynamics.

Thin ctypes binding of libmdjump.so, whose C ABI is include/md.h. Every step
of the hot path runs in the library's CUDA kernels; this module only marshals
arguments. Importing it does not need a GPU; creating an Engine does, and it
fails loudly when the compiled library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import systems  # noqa: F401  (input builders)

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmdjump.so")

MD_FP64, MD_MIXED = 0, 1
GRAD_FULL, GRAD_BONDED, GRAD_NB_FULL, GRAD_NB_SHORT, GRAD_NB_LONG, GRAD_F0, GRAD_RECIP = range(7)
COULOMB_DSF, COULOMB_EWALD = 0, 1
N_PROFILE_CLASSES = 9
FLAG_BOUND, FLAG_LIMIT, FLAG_NONFINITE, FLAG_OVERFLOW = 1, 2, 4, 8
ERRORS = {-1: "MD_EINVAL", -2: "MD_ECUDA", -3: "MD_EOVERFLOW", -4: "MD_EBOUND",
          -5: "MD_ELIMIT", -6: "MD_ENONFINITE", -7: "MD_ENOSYSTEM", -8: "MD_ENOMEM"}

# exported symbols of include/md.h
SYMBOLS = ["md_init", "md_set_system", "md_set_state", "md_step_baoab", "md_step_baoab_respa",
           "md_step_baoab_respa1", "md_step_jump", "md_step_bjaoajb", "md_step_jump_respa", "md_step_jump_respa1",
           "md_observables", "md_get_state", "md_gradient", "md_run_phase", "md_get_list",
           "md_get_events", "md_profile", "md_vacf_start", "md_vacf_get", "md_nb_gradient_noalloc",
           "md_finalize", "md_last_error"]


class MDError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class MdConfig(C.Structure):
    _fields_ = [("precision", C.c_int), ("seed", C.c_uint64), ("device", C.c_int),
                ("cuda_stream", C.c_void_p), ("max_replicas", C.c_int),
                ("event_log_cap", C.c_int64), ("threads_per_atom", C.c_int), ("no_graphs", C.c_int)]


class MdSystem(C.Structure):
    _fields_ = [("n_atoms", C.c_int), ("box", C.c_double),
                ("x", C.c_void_p), ("v", C.c_void_p), ("mass", C.c_void_p), ("charge", C.c_void_p),
                ("type", C.c_void_p), ("n_types", C.c_int), ("lj_eps", C.c_void_p),
                ("lj_sigma", C.c_void_p),
                ("n_bonds", C.c_int), ("bonds", C.c_void_p), ("bond_k", C.c_void_p), ("bond_r0", C.c_void_p),
                ("n_angles", C.c_int), ("angles", C.c_void_p), ("angle_k", C.c_void_p),
                ("angle_t0", C.c_void_p),
                ("n_excl", C.c_int), ("excl_pairs", C.c_void_p),
                ("r_cut", C.c_double), ("r_split", C.c_double), ("h_switch", C.c_double),
                ("r_mid", C.c_double), ("dsf_alpha", C.c_double), ("gamma", C.c_double),
                ("temperature", C.c_double), ("eps0", C.c_double), ("eps_mode", C.c_int),
                ("skin", C.c_double), ("skin_outer", C.c_double),
                ("n_rings", C.c_int), ("ring_r", C.c_double * 3), ("lj_long_mode", C.c_int),
                ("coulomb_mode", C.c_int), ("pme_order", C.c_int), ("pme_spacing", C.c_double)]


class MdObs(C.Structure):
    _fields_ = [("ke", C.c_double), ("temperature", C.c_double), ("pe_bond", C.c_double),
                ("pe_angle", C.c_double), ("pe_lj", C.c_double), ("pe_coul", C.c_double),
                ("step", C.c_int64), ("jump_proposals", C.c_int64), ("jump_accepts", C.c_int64),
                ("bps_proposals", C.c_int64), ("bps_accepts", C.c_int64),
                ("sampler_attempts", C.c_int64), ("list_rebuilds", C.c_int64),
                ("outer_rebuilds", C.c_int64), ("guarded_accepts", C.c_int64),
                ("error_flags", C.c_uint32)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libmdjump.so and declare its C ABI. Raises if it is not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    L = C.CDLL(path)
    P, vp, i, d, i64 = C.POINTER, C.c_void_p, C.c_int, C.c_double, C.c_int64
    L.md_init.argtypes = [P(vp), P(MdConfig)]
    L.md_set_system.argtypes = [vp, i, P(MdSystem)]
    L.md_set_state.argtypes = [vp, i, vp, vp, vp, vp, vp, i64]
    for n in ("md_step_baoab", "md_step_jump", "md_step_bjaoajb"):
        getattr(L, n).argtypes = [vp, i64, d]
    for n in ("md_step_baoab_respa", "md_step_jump_respa"):
        getattr(L, n).argtypes = [vp, i64, d, i]
    for n in ("md_step_baoab_respa1", "md_step_jump_respa1"):
        getattr(L, n).argtypes = [vp, i64, d, i, i]
    L.md_observables.argtypes = [vp, i, P(MdObs)]
    L.md_get_state.argtypes = [vp, i, vp, vp, vp, vp, vp]
    L.md_gradient.argtypes = [vp, i, i, vp]
    L.md_run_phase.argtypes = [vp, i, d, i64, i, i]
    L.md_get_list.argtypes = [vp, i, i, i, vp, i]
    L.md_get_events.restype = i64
    L.md_get_events.argtypes = [vp, i, vp, i64, i]
    L.md_profile.argtypes = [vp, i, i, vp, vp, vp]
    L.md_vacf_start.argtypes = [vp, i64]
    L.md_vacf_get.argtypes = [vp, i, i64, vp, vp, P(C.c_int64)]
    L.md_nb_gradient_noalloc.argtypes = [vp, vp, vp, vp, i, d, i, vp, vp, d, d, d, d, i, vp, vp]
    L.md_finalize.argtypes = [vp]
    L.md_last_error.restype = C.c_char_p
    L.md_last_error.argtypes = [vp]
    _lib = L
    return L


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


DEFAULTS = dict(r_cut=9.0, r_split=5.0, h_switch=0.5, r_mid=5.5, dsf_alpha=0.2, gamma=1.0,
                temperature=300.0, eps0=0.1, eps_mode=1, skin=0.3, skin_outer=None, ring_r=None, lj_long_mode=0,
                coulomb_mode=0, pme_order=6, pme_spacing=0.8)


KIND_RING0, KIND_LJ = 0, 4


class Engine:
    """One md_ctx: a batch of replicas advanced together on one GPU."""

    def __init__(self, precision=MD_MIXED, seed=0, device=0, stream=None, max_replicas=1,
                 event_log_cap=0, threads_per_atom=0, graphs=True):
        self.L = load_library()
        if stream is None:
            stream = _current_stream()
        self.cfg = MdConfig(precision, seed, device, stream, max_replicas, event_log_cap, threads_per_atom,
                            0 if graphs else 1)
        h = C.c_void_p()
        rc = self.L.md_init(C.byref(h), C.byref(self.cfg))
        if rc != 0:
            raise MDError(rc, self.L.md_last_error(None).decode())
        self.h = h
        self.n = {}

    def _ck(self, rc):
        if rc < 0:
            raise MDError(rc, self.L.md_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            self.L.md_finalize(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_system(self, replica, sys, **kw):
        p = dict(DEFAULTS)
        p.update(kw)
        if p["skin_outer"] is None:
            p["skin_outer"] = p["skin"]
        a = lambda z, t: np.ascontiguousarray(z, dtype=t)
        keep = dict(x=a(sys.x, np.float64), v=a(sys.v, np.float64), mass=a(sys.mass, np.float64),
                    charge=a(sys.charge, np.float64), type=a(sys.type, np.int32),
                    lj_eps=a(sys.lj_eps, np.float64), lj_sigma=a(sys.lj_sigma, np.float64),
                    bonds=a(sys.bonds, np.int32), bond_k=a(sys.bond_k, np.float64),
                    bond_r0=a(sys.bond_r0, np.float64), angles=a(sys.angles, np.int32),
                    angle_k=a(sys.angle_k, np.float64), angle_t0=a(sys.angle_t0, np.float64),
                    excl=a(sys.excl, np.int32))
        # the library reads these through plain pointers: check their sizes here
        n, nt = int(sys.n), int(keep["lj_eps"].shape[0])
        sizes = dict(x=3 * n, v=3 * n, mass=n, charge=n, type=n, lj_eps=nt * nt, lj_sigma=nt * nt,
                     bonds=2 * len(keep["bond_k"]), bond_r0=len(keep["bond_k"]),
                     angles=3 * len(keep["angle_k"]), angle_t0=len(keep["angle_k"]),
                     excl=2 * int(keep["excl"].shape[0]))
        for name, want in sizes.items():
            if keep[name].size != want:
                raise ValueError(f"set_system: {name} has {keep[name].size} values, expected {want}")
        s = MdSystem(sys.n, sys.box, _ptr(keep["x"]), _ptr(keep["v"]), _ptr(keep["mass"]),
                     _ptr(keep["charge"]), _ptr(keep["type"]), int(sys.lj_eps.shape[0]),
                     _ptr(keep["lj_eps"]), _ptr(keep["lj_sigma"]), len(sys.bond_k), _ptr(keep["bonds"]),
                     _ptr(keep["bond_k"]), _ptr(keep["bond_r0"]), len(sys.angle_k), _ptr(keep["angles"]),
                     _ptr(keep["angle_k"]), _ptr(keep["angle_t0"]), int(sys.excl.shape[0]),
                     _ptr(keep["excl"]), p["r_cut"], p["r_split"], p["h_switch"], p["r_mid"],
                     p["dsf_alpha"], p["gamma"], p["temperature"], p["eps0"], p["eps_mode"],
                     p["skin"], p["skin_outer"])
        # ring_r: interior ring edges; None keeps the rings of r_mid
        if p["ring_r"] is not None:
            rr = [float(z) for z in p["ring_r"]]
            if len(rr) > 3:
                raise ValueError("at most 3 interior ring edges (4 rings)")
            s.n_rings = len(rr) + 1
            for k, z in enumerate(rr):
                s.ring_r[k] = z
        s.lj_long_mode = int(p["lj_long_mode"])
        s.coulomb_mode = int(p["coulomb_mode"])
        s.pme_order = int(p["pme_order"])
        s.pme_spacing = float(p["pme_spacing"])
        self._ck(self.L.md_set_system(self.h, replica, C.byref(s)))
        self.n[replica] = sys.n

    def set_state(self, replica, x, v, img=None, x_build=None, x_outer=None, step=0):
        f = lambda z, t: None if z is None else np.ascontiguousarray(z, dtype=t)
        x, v, img, xb, xo = f(x, np.float64), f(v, np.float64), f(img, np.int32), f(x_build, np.float64), f(x_outer, np.float64)
        n3 = 3 * self.n[replica]
        for name, z in (("x", x), ("v", v), ("img", img), ("x_build", xb), ("x_outer", xo)):
            if z is not None and z.size != n3:
                raise ValueError(f"set_state: {name} has {z.size} values, expected {n3}")
        self._ck(self.L.md_set_state(self.h, replica, _ptr(x), _ptr(v), _ptr(img), _ptr(xb), _ptr(xo), int(step)))

    def baoab(self, nsteps, dt_fs=1.0):
        return self._ck(self.L.md_step_baoab(self.h, int(nsteps), float(dt_fs)))

    def jump(self, nsteps, dt_fs=1.0):
        return self._ck(self.L.md_step_jump(self.h, int(nsteps), float(dt_fs)))

    def bjaoajb(self, nsteps, dt_fs=1.0):
        return self._ck(self.L.md_step_bjaoajb(self.h, int(nsteps), float(dt_fs)))

    def baoab_respa(self, n_outer, dt_inner_fs=1.0, n_inner=2):
        return self._ck(self.L.md_step_baoab_respa(self.h, int(n_outer), float(dt_inner_fs), int(n_inner)))

    def jump_respa(self, n_outer, dt_inner_fs=1.0, n_inner=2):
        return self._ck(self.L.md_step_jump_respa(self.h, int(n_outer), float(dt_inner_fs), int(n_inner)))

    def baoab_respa1(self, n_outer, dt_inner_fs=1.0, m_mid=2, n_outer_ratio=2):
        return self._ck(self.L.md_step_baoab_respa1(self.h, int(n_outer), float(dt_inner_fs), int(m_mid), int(n_outer_ratio)))

    def jump_respa1(self, n_outer, dt_inner_fs=1.0, m_mid=2, n_outer_ratio=2):
        return self._ck(self.L.md_step_jump_respa1(self.h, int(n_outer), float(dt_inner_fs), int(m_mid), int(n_outer_ratio)))

    def observables(self, replica=0) -> dict:
        o = MdObs()
        self._ck(self.L.md_observables(self.h, replica, C.byref(o)))
        return {k: getattr(o, k) for k, _ in MdObs._fields_}

    def state(self, replica=0, outer=False):
        n = self.n[replica]
        x, v, xb, xo = (np.zeros((n, 3)) for _ in range(4))
        img = np.zeros((n, 3), dtype=np.int32)
        self._ck(self.L.md_get_state(self.h, replica, _ptr(x), _ptr(v), _ptr(img), _ptr(xb), _ptr(xo)))
        return (x, v, img, xb, xo) if outer else (x, v, img, xb)

    def gradient(self, mode=GRAD_FULL, replica=0):
        g = np.zeros((self.n[replica], 3))
        self._ck(self.L.md_gradient(self.h, replica, mode, _ptr(g)))
        return g

    def run_phase(self, phase, tau2_ps, s0, half, accel_mode=GRAD_F0):
        self._ck(self.L.md_run_phase(self.h, int(phase), float(tau2_ps), int(s0), int(half), int(accel_mode)))

    def get_list(self, kind, atom, replica=0, cap=4096):
        """Jump list of one atom: kind 0..3 ring 0..3 (inner to outer), 4 LJ."""
        out = np.zeros(cap, dtype=np.int32)
        n = self._ck(self.L.md_get_list(self.h, replica, kind, atom, _ptr(out), cap))
        return out[:min(n, cap)]

    def profile(self, enable=-1, reset=False):
        """(ms per class, timed groups per class, kernels launched per class);
        classes: pair force, bonded, velocity phases, kicks/AOA, list cells and outer candidates,
        bookkeeping, Ewald reciprocal (PME), inner list filter, rate ordering."""
        ms = np.zeros(N_PROFILE_CLASSES)
        groups = np.zeros(N_PROFILE_CLASSES, dtype=np.int64)
        launches = np.zeros(N_PROFILE_CLASSES, dtype=np.int64)
        self._ck(self.L.md_profile(self.h, int(enable), int(reset), _ptr(ms), _ptr(groups), _ptr(launches)))
        return ms, groups, launches

    def vacf_start(self, n_samples):
        """record v after every innermost step (n_samples steps at most; 0 ends the record)"""
        self._ck(self.L.md_vacf_start(self.h, int(n_samples)))

    def vacf(self, n_lags, replica=0):
        """(mass-weighted VACF C(k), its Hann-windowed cosine transform S(j), samples stored)"""
        c = np.zeros(int(n_lags))
        sp = np.zeros(int(n_lags))
        t = C.c_int64(0)
        self._ck(self.L.md_vacf_get(self.h, replica, int(n_lags), _ptr(c), _ptr(sp), C.byref(t)))
        return c, sp, t.value

    def events(self, replica=0, cap=1 << 22, clear=True) -> np.ndarray:
        out = np.zeros((cap, 6), dtype=np.int64)
        n = self._ck(self.L.md_get_events(self.h, replica, _ptr(out), cap, int(clear)))
        return out[:n]
