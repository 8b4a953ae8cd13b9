"""ctypes front end of the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference leg may import this package. It shares no code with
the CUDA path: it reads systems built by paper_2412_15073_gb300.systems (pure
input generation) and calls liboracle.so, compiled from oracle.c by build().
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle.so")
# a library built elsewhere from an edited oracle.c (the planted-mistake
# checks of tests/test_oracle_mutations.py); never set in normal use
EXTERNAL_LIB = os.environ.get("ORACLE_MUTANT_LIB")
if EXTERNAL_LIB:
    LIB = EXTERNAL_LIB
CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off"]

GRAD_FULL, GRAD_BONDED, GRAD_NB_FULL, GRAD_NB_SHORT, GRAD_NB_LONG, GRAD_F0 = range(6)
KIND_RING_M, KIND_RING_L, KIND_LJ = 0, 1, 4     # ring y is kind y (0..3); LJ partners kind 4
E_BOUND, E_LIMIT, E_NONFIN = 1, 2, 4


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (FP contraction off, OpenMP on)."""
    if EXTERNAL_LIB:
        return LIB
    src = os.path.join(HERE, "oracle.c")
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(src),
                                             os.path.getmtime(os.path.join(HERE, "oracle.h")))):
        return LIB
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", *CFLAGS, "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


class Params(C.Structure):
    _fields_ = [("box", C.c_double), ("r_cut", C.c_double), ("r_split", C.c_double),
                ("h_switch", C.c_double), ("r_mid", C.c_double), ("dsf_alpha", C.c_double),
                ("gamma", C.c_double), ("temperature", C.c_double), ("eps0", C.c_double),
                ("skin", C.c_double), ("skin_outer", C.c_double), ("eps_mode", C.c_int),
                ("n_rings", C.c_int), ("ring_r", C.c_double * 3), ("seed", C.c_uint32),
                ("replica", C.c_uint32), ("lazy_lists", C.c_int), ("lj_long_mode", C.c_int),
                ("coulomb_mode", C.c_int), ("pme_order", C.c_int), ("pme_spacing", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        P = C.POINTER
        d, i, i64, u32 = C.c_double, C.c_int, C.c_int64, C.c_uint32
        vp = C.c_void_p
        L.or_create.restype = vp
        L.or_create.argtypes = [i, P(Params), vp, vp, vp, vp, vp, i, vp, vp, i, vp, vp, vp,
                                i, vp, vp, vp, i, vp]
        L.or_destroy.argtypes = [vp]
        L.or_ewald_recip_plain.argtypes = [vp, i, vp, vp]
        L.or_ewald_recip_pme.argtypes = [vp, vp, vp, vp]
        L.or_set_threads.argtypes = [i]
        L.or_get_threads.restype = i
        L.or_get_state.argtypes = [vp, vp, vp, vp, vp, vp]
        L.or_set_state.argtypes = [vp, vp, vp, vp, vp, vp, i64]
        L.or_step_count.restype = i64
        L.or_step_count.argtypes = [vp]
        L.or_counters.argtypes = [vp, vp]
        L.or_errors.restype = u32
        L.or_errors.argtypes = [vp]
        L.or_gradient.argtypes = [vp, i, vp, vp]
        L.or_gradient_atom.argtypes = [vp, i, i, vp]
        L.or_energy.argtypes = [vp, vp]
        L.or_bounds.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.or_list_counts.argtypes = [vp, i, vp]
        L.or_list_get.restype = i
        L.or_list_get.argtypes = [vp, i, i, vp]
        L.or_rebuild.argtypes = [vp]
        L.or_cprime_one.argtypes = [vp, i, vp, vp, d, u32, i, vp, vp, vp]
        L.or_jprime_one.argtypes = [vp, i, vp, d, u32, i, vp, vp, vp]
        L.or_sample_atom_work.restype = i
        L.or_sample_atom_work.argtypes = [vp, i, vp, i, i, i, d, u32, i]
        for name in ("or_step_baoab", "or_step_jump", "or_step_bjaoajb"):
            getattr(L, name).restype = i
            getattr(L, name).argtypes = [vp, i64, d]
        for name in ("or_step_baoab_respa", "or_step_jump_respa"):
            getattr(L, name).restype = i
            getattr(L, name).argtypes = [vp, i64, d, i]
        for name in ("or_step_baoab_respa1", "or_step_jump_respa1"):
            getattr(L, name).restype = i
            getattr(L, name).argtypes = [vp, i64, d, i, i]
        L.or_events_enable.argtypes = [vp, i64]
        L.or_events_get.restype = i64
        L.or_events_get.argtypes = [vp, vp]
        L.or_vrec_enable.argtypes = [vp, i64]
        L.or_vrec_get.restype = i64
        L.or_vrec_get.argtypes = [vp, vp]
        L.or_vacf.argtypes = [vp, vp, i, i64, i64, vp]
        L.or_vacf_spectrum.argtypes = [vp, i64, vp]
        L.or_philox.argtypes = [vp, vp, vp]
        L.or_theta.restype = d
        L.or_theta.argtypes = [d]
        L.or_sample_gtilde.restype = d
        L.or_sample_gtilde.argtypes = [d, u32, u32, u32, u32, i, u32, P(C.c_int)]
        L.or_pair_dudr.restype = d
        L.or_pair_dudr.argtypes = [vp, i, i, d, d, i]
        L.or_pair_u.restype = d
        L.or_pair_u.argtypes = [vp, i, i, d, d, i]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox(_p(c), _p(k), _p(out))
    return out


def theta(eta: float) -> float:
    return lib().or_theta(float(eta))


def sample_gtilde(eta, seed=0, replica=0, atom=0, s0=0, half=0, k=0):
    att = C.c_int(0)
    y = lib().or_sample_gtilde(float(eta), seed, replica, atom, s0, half, k, C.byref(att))
    return y, att.value


class Oracle:
    """One system advanced by the oracle. `sys` is a systems.System."""

    def __init__(self, sys, r_cut=9.0, r_split=5.0, h_switch=0.5, r_mid=5.5, dsf_alpha=0.2,
                 gamma=1.0, temperature=300.0, eps0=0.1, skin=0.3, skin_outer=None, eps_mode=1,
                 seed=0, replica=0, ring_r=None, lazy_lists=False, lj_long_mode=0,
                 coulomb_mode=0, pme_order=6, pme_spacing=0.8):
        self.L = lib()
        self.n = sys.n
        if skin_outer is None:
            skin_outer = skin
        if coulomb_mode == 1 and pme_order not in (4, 6, 8):
            raise ValueError("pme_order must be 4, 6 or 8 (an odd order has b(m) = 0 at m = K/2 on even grids)")
        rr = list(ring_r or [])
        n_rings = len(rr) + 1 if ring_r is not None else 0
        self.params = Params(sys.box, r_cut, r_split, h_switch, r_mid, dsf_alpha, gamma,
                             temperature, eps0, skin, skin_outer, eps_mode, n_rings,
                             (C.c_double * 3)(*(rr + [0.0] * (3 - len(rr)))), seed, replica,
                             1 if lazy_lists else 0, int(lj_long_mode), int(coulomb_mode), int(pme_order),
                             float(pme_spacing))
        a = lambda z, t: np.ascontiguousarray(z, dtype=t)
        self._keep = [a(sys.x, np.float64), a(sys.v, np.float64), a(sys.mass, np.float64),
                      a(sys.charge, np.float64), a(sys.type, np.int32), a(sys.lj_eps, np.float64),
                      a(sys.lj_sigma, np.float64), a(sys.bonds, np.int32), a(sys.bond_k, np.float64),
                      a(sys.bond_r0, np.float64), a(sys.angles, np.int32), a(sys.angle_k, np.float64),
                      a(sys.angle_t0, np.float64), a(sys.excl, np.int32)]
        k = self._keep
        self.h = self.L.or_create(self.n, C.byref(self.params), _p(k[0]), _p(k[1]), _p(k[2]),
                                  _p(k[3]), _p(k[4]), int(sys.lj_eps.shape[0]), _p(k[5]), _p(k[6]),
                                  len(sys.bond_k), _p(k[7]), _p(k[8]), _p(k[9]),
                                  len(sys.angle_k), _p(k[10]), _p(k[11]), _p(k[12]),
                                  int(sys.excl.shape[0]), _p(k[13]))

    def __del__(self):
        if getattr(self, "h", None):
            self.L.or_destroy(self.h)
            self.h = None

    # state ---------------------------------------------------------------
    def state(self, outer=False):
        x = np.zeros((self.n, 3)); v = np.zeros((self.n, 3))
        img = np.zeros((self.n, 3), dtype=np.int32); xb = np.zeros((self.n, 3))
        xo = np.zeros((self.n, 3))
        self.L.or_get_state(self.h, _p(x), _p(v), _p(img), _p(xb), _p(xo))
        return (x, v, img, xb, xo) if outer else (x, v, img, xb)

    def set_state(self, x, v, img=None, x_build=None, step=0, x_outer=None):
        f = lambda z, t: None if z is None else np.ascontiguousarray(z, dtype=t)
        x, v, img = f(x, np.float64), f(v, np.float64), f(img, np.int32)
        xb, xo = f(x_build, np.float64), f(x_outer, np.float64)
        q = lambda z: None if z is None else _p(z)
        self.L.or_set_state(self.h, _p(x), _p(v), q(img), q(xb), q(xo), int(step))

    @property
    def step(self) -> int:
        return self.L.or_step_count(self.h)

    def counters(self) -> np.ndarray:
        out = np.zeros(6, dtype=np.int64)
        self.L.or_counters(self.h, _p(out))
        return out

    @property
    def errors(self) -> int:
        return self.L.or_errors(self.h)

    # forces --------------------------------------------------------------
    def gradient(self, mode=GRAD_FULL):
        g = np.zeros((self.n, 3)); e = C.c_double(0)
        self.L.or_gradient(self.h, mode, _p(g), C.byref(e))
        return g, e.value

    def gradient_atom(self, mode, i):
        g = np.zeros(3)
        self.L.or_gradient_atom(self.h, mode, int(i), _p(g))
        return g

    def energy(self) -> np.ndarray:
        t = np.zeros(4)
        self.L.or_energy(self.h, _p(t))
        return t

    def pair_dudr(self, ti, tj, qiqj, r, weight=0):
        return self.L.or_pair_dudr(self.h, ti, tj, float(qiqj), float(r), weight)

    def pair_u(self, ti, tj, qiqj, r, weight=0):
        return self.L.or_pair_u(self.h, ti, tj, float(qiqj), float(r), weight)

    def bounds(self):
        """(lhat[4], qmax, ring edges, n_rings, LY (n x 4), LLJ (n))"""
        lhat = np.zeros(4); q = np.zeros(1); edges = np.zeros(5); nr = C.c_int(0)
        LY = np.zeros((self.n, 4)); LJ = np.zeros(self.n)
        self.L.or_bounds(self.h, _p(lhat), _p(q), _p(edges), C.byref(nr), _p(LY), _p(LJ))
        return lhat, float(q[0]), edges[:nr.value + 1], nr.value, LY, LJ

    # lists ---------------------------------------------------------------
    def list_counts(self, kind):
        c = np.zeros(self.n, dtype=np.int32)
        self.L.or_list_counts(self.h, kind, _p(c))
        return c

    def list_of(self, kind, i):
        out = np.zeros(max(self.n, 1), dtype=np.int32)          # a list never exceeds the atom count
        m = self.L.or_list_get(self.h, kind, int(i), _p(out))
        return out[:m]

    def rebuild(self):
        self.L.or_rebuild(self.h)

    # phases --------------------------------------------------------------
    def cprime_one(self, i, v, a, tau2, s0, half):
        v = np.ascontiguousarray(v, dtype=np.float64); a = np.ascontiguousarray(a, dtype=np.float64)
        out = np.zeros(3); np_ = C.c_int64(0); na = C.c_int64(0)
        self.L.or_cprime_one(self.h, int(i), _p(v), _p(a), float(tau2), int(s0), int(half),
                             _p(out), C.byref(np_), C.byref(na))
        return out, np_.value, na.value

    def jprime_one(self, i, v, tau2, s0, half):
        v = np.ascontiguousarray(v, dtype=np.float64)
        out = np.zeros(3); np_ = C.c_int64(0); na = C.c_int64(0)
        self.L.or_jprime_one(self.h, int(i), _p(v), float(tau2), int(s0), int(half),
                             _p(out), C.byref(np_), C.byref(na))
        return out, np_.value, na.value

    def sample_atom_work(self, atoms, mode, n_grad, n_phase, tau2, s0, nthreads):
        """timing workload of the CPU baseline (see or_sample_atom_work); returns the threads used"""
        a = np.ascontiguousarray(atoms, dtype=np.int32)
        return self.L.or_sample_atom_work(self.h, len(a), _p(a), int(mode), int(n_grad), int(n_phase),
                                          float(tau2), int(s0), int(nthreads))

    # integrators ---------------------------------------------------------
    def baoab(self, nsteps, dt_fs=1.0):
        return self.L.or_step_baoab(self.h, int(nsteps), float(dt_fs))

    def jump(self, nsteps, dt_fs=1.0):
        return self.L.or_step_jump(self.h, int(nsteps), float(dt_fs))

    def ewald_recip_plain(self, kmax):
        """(gradient n x 3, energy) of the reciprocal part by the plain Ewald sum (+ self, exclusions)"""
        g = np.zeros((self.n, 3))
        e = C.c_double(0.0)
        self.L.or_ewald_recip_plain(self.h, int(kmax), _p(g), C.byref(e))
        return g, e.value

    def ewald_recip_pme(self):
        """(gradient n x 3, energy, K) of the reciprocal part by smooth PME (+ self, exclusions)"""
        g = np.zeros((self.n, 3))
        e = C.c_double(0.0)
        K = C.c_int(0)
        self.L.or_ewald_recip_pme(self.h, _p(g), C.byref(e), C.byref(K))
        return g, e.value, K.value

    def bjaoajb(self, nsteps, dt_fs=1.0):
        return self.L.or_step_bjaoajb(self.h, int(nsteps), float(dt_fs))

    def baoab_respa(self, nouter, dt_inner_fs=1.0, n_inner=2):
        return self.L.or_step_baoab_respa(self.h, int(nouter), float(dt_inner_fs), int(n_inner))

    def jump_respa(self, nouter, dt_inner_fs=1.0, n_inner=2):
        return self.L.or_step_jump_respa(self.h, int(nouter), float(dt_inner_fs), int(n_inner))

    def baoab_respa1(self, nouter, dt_inner_fs=1.0, m_mid=2, n_outer=2):
        return self.L.or_step_baoab_respa1(self.h, int(nouter), float(dt_inner_fs), int(m_mid), int(n_outer))

    def jump_respa1(self, nouter, dt_inner_fs=1.0, m_mid=2, n_outer=2):
        return self.L.or_step_jump_respa1(self.h, int(nouter), float(dt_inner_fs), int(m_mid), int(n_outer))

    # velocity record -----------------------------------------------------
    def vrec_enable(self, cap):
        self.L.or_vrec_enable(self.h, int(cap))

    def vrec(self) -> np.ndarray:
        """the stored velocities, T x n x 3"""
        T = self.L.or_vrec_get(self.h, None)
        out = np.zeros((max(T, 1), self.n, 3))
        self.L.or_vrec_get(self.h, _p(out))
        return out[:T]

    # events --------------------------------------------------------------
    def events_enable(self, cap=1 << 20):
        self.L.or_events_enable(self.h, int(cap))

    def events(self) -> np.ndarray:
        n = self.L.or_events_get(self.h, None)
        out = np.zeros((max(n, 1), 6), dtype=np.int64)
        self.L.or_events_get(self.h, _p(out))
        return out[:n]


def vacf(v, mass, nlags):
    """Mass-weighted velocity autocorrelation of a series v[T, n, 3] (or[T, 3n])
    by its definition: C(k) = sum_t sum_i m_i v_i(t).v_i(t+k) / (T - k)."""
    mass = np.ascontiguousarray(mass, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1, len(mass) * 3)
    out = np.zeros(int(nlags))
    lib().or_vacf(_p(v), _p(mass), len(mass), v.shape[0], int(nlags), _p(out))
    return out


def vacf_spectrum(C):
    """Hann-windowed cosine transform of an autocorrelation (see or_vacf_spectrum)."""
    C = np.ascontiguousarray(C, dtype=np.float64)
    S = np.zeros(len(C))
    lib().or_vacf_spectrum(_p(C), len(C), _p(S))
    return S


def set_threads(n: int):
    lib().or_set_threads(int(n))


def get_threads() -> int:
    return lib().or_get_threads()
