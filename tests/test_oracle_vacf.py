"""The oracle's velocity record and autocorrelation (the spectra of Sec. 4):
the VACF of a pure cosine against its closed form, random series against
numpy's correlation, the windowed cosine transform on series whose spectrum
is known, and the places where the integrators take their samples."""
import numpy as np
import pytest

from paper_2412_15073_gb300 import systems

PARAMS = dict(r_cut=9.0, r_split=5.0, h_switch=0.5, r_mid=5.5, dsf_alpha=0.2, gamma=1.0,
              temperature=300.0, eps0=0.1, eps_mode=1, skin=0.2, skin_outer=0.3)


def test_vacf_of_a_cosine_matches_its_closed_form(oracle_mod):
    """v(t) = A cos(w t + phi) along x for one atom of mass m: by the product
    to sum rule and the Dirichlet sum sum_{t<M} cos(a + 2 w t) =
    sin(M w) cos(a + (M - 1) w) / sin(w),
    C(k) = m A^2 / 2 [cos(w k) + sin(M w) cos(w k + 2 phi + (M - 1) w) / (M sin w)], M = T - k"""
    T, m, A, w, phi = 240, 2.5, 1.7, 0.37, 0.4
    t = np.arange(T)
    v = np.zeros((T, 1, 3))
    v[:, 0, 0] = A * np.cos(w * t + phi)
    C = oracle_mod.vacf(v, [m], 60)
    k = np.arange(60)
    M = T - k
    ref = 0.5 * m * A * A * (np.cos(w * k) + np.sin(M * w) * np.cos(w * k + 2 * phi + (M - 1) * w) / (M * np.sin(w)))
    np.testing.assert_allclose(C, ref, rtol=1e-12, atol=1e-12)


def test_vacf_of_random_series_matches_numpy_correlate(oracle_mod):
    rng = np.random.default_rng(4)
    T, n = 50, 4
    v = rng.normal(size=(T, n, 3))
    mass = rng.uniform(1, 16, size=n)
    C = oracle_mod.vacf(v, mass, 70)
    ref = np.zeros(70)
    for i in range(n):
        for c in range(3):
            full = np.correlate(v[:, i, c], v[:, i, c], mode="full")[T - 1:]    # sum_t x(t) x(t + k)
            ref[:T] += mass[i] * full
    ref[:T] /= T - np.arange(T)
    np.testing.assert_allclose(C, ref, rtol=1e-12, atol=1e-12)
    assert (C[T:] == 0).all()


def test_windowed_spectrum_on_known_autocorrelations(oracle_mod):
    K = 256
    # white noise: C = delta -> flat spectrum
    d = np.zeros(K)
    d[0] = 3.0
    np.testing.assert_allclose(oracle_mod.vacf_spectrum(d), 3.0, rtol=0, atol=1e-12)
    # a cosine at bin j0 (frequency j0 / (2 K dt)): the spectrum peaks there and
    # holds about K/2 of weight at the peak (window sum 1 + (K - 1) / 2)
    for j0 in (20, 77):
        S = oracle_mod.vacf_spectrum(np.cos(np.pi * j0 * np.arange(K) / K))
        assert int(np.argmax(S)) == j0
        assert S[j0] == pytest.approx(0.5 * K + 0.5, rel=1e-2)
        assert abs(S[j0 + 8]) < 1e-2 * S[j0]
    # linearity
    a, b = np.random.default_rng(1).normal(size=(2, K))
    np.testing.assert_allclose(oracle_mod.vacf_spectrum(2 * a - b),
                               2 * oracle_mod.vacf_spectrum(a) - oracle_mod.vacf_spectrum(b), atol=1e-9)


def _record(oracle_mod, w, integ, args, cap):
    o = oracle_mod.Oracle(w, seed=2, **PARAMS)
    o.vrec_enable(cap)
    getattr(o, integ)(*args)
    return o.vrec()


def test_record_places_follow_the_integrator_identities(oracle_mod):
    """one sample per innermost step; RESPA with one inner step is BAOAB (up to
    the rounding of kicking the bonded and nonbonded parts apart), and with DSF
    (no outer force) JUMP-RESPA1 is JUMP-RESPA at the mid level, so their
    records coincide sample for sample"""
    w = systems.water_box(27, box=18.643, seed=0)
    a = _record(oracle_mod, w, "baoab", (12,), 100)
    b = _record(oracle_mod, w, "baoab_respa", (12, 1.0, 1), 100)
    assert a.shape == (12, 81, 3)
    np.testing.assert_allclose(a, b, rtol=1e-10, atol=1e-10)
    c = _record(oracle_mod, w, "jump_respa", (6, 1.0, 2), 100)
    d = _record(oracle_mod, w, "jump_respa1", (3, 1.0, 2, 2), 100)
    assert c.shape == (12, 81, 3)
    np.testing.assert_array_equal(c, d)
    # the cap keeps the first samples
    e = _record(oracle_mod, w, "baoab", (12,), 5)
    np.testing.assert_array_equal(e, a[:5])
    # the last sample is the state the step call leaves
    o = oracle_mod.Oracle(w, seed=2, **PARAMS)
    o.vrec_enable(100)
    o.baoab_respa1(2, 1.0, 2, 3)
    np.testing.assert_array_equal(o.vrec()[-1], o.state()[1])
    assert len(o.vrec()) == 12
