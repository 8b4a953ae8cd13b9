"""Velocity record and autocorrelation spectra on the GPU (md_vacf_start /
md_vacf_get) against the oracle's record and its VACF by definition."""
import numpy as np
import pytest

from test_gpu_parity import PARAMS

pytestmark = pytest.mark.gpu

EWALD = dict(dsf_alpha=0.35, coulomb_mode=1, pme_order=6, pme_spacing=0.8)


@pytest.fixture(scope="module")
def M():
    import paper_2412_15073_gb300 as M
    M.load_library()
    return M


@pytest.mark.parametrize("integ,args,kw", [
    ("baoab", (60,), {}),
    ("jump", (60,), {}),
    ("jump_respa1", (15, 1.0, 2, 2), {}),
    ("baoab_respa1", (10, 1.0, 2, 3), EWALD),
    ("jump_respa1", (10, 1.0, 2, 3), EWALD),
])
def test_fp64_record_and_vacf_match_the_oracle(M, oracle_mod, water648, integ, args, kw):
    p = PARAMS | kw
    e = M.Engine(precision=M.MD_FP64, seed=9)
    e.set_system(0, water648, **p)
    o = oracle_mod.Oracle(water648, seed=9, **p)
    e.vacf_start(200)
    o.vrec_enable(200)
    getattr(e, integ)(*args)
    getattr(o, integ)(*args)
    K = 48
    C, S, T = e.vacf(K)
    series = o.vrec()
    assert T == len(series) == 60
    Co = oracle_mod.vacf(series, water648.mass, K)
    So = oracle_mod.vacf_spectrum(Co)
    np.testing.assert_allclose(C, Co, rtol=1e-6)
    np.testing.assert_allclose(S, So, rtol=0, atol=1e-6 * np.abs(So).max())


def test_mixed_record_equals_the_states_of_single_steps(M, oracle_mod, water648):
    """mixed precision: the record of one 64-step call (CUDA graphs) and of 64
    one-step calls are the same, and the VACF equals the oracle's definition
    applied to the states md_get_state returned after each step (FP32 record)"""
    K = 40
    outs = []
    for single in (True, False):
        e = M.Engine(precision=M.MD_MIXED, seed=4)
        e.set_system(0, water648, **PARAMS)
        e.vacf_start(64)
        host = []
        if single:
            for _ in range(64):
                e.jump(1)
                host.append(e.state()[1])
        else:
            e.jump(64)
        outs.append(e.vacf(K))
        if single:
            Co = oracle_mod.vacf(np.stack(host), water648.mass, K)
    (C1, S1, T1), (C2, S2, T2) = outs
    assert T1 == T2 == 64
    np.testing.assert_array_equal(C1, C2)
    np.testing.assert_array_equal(S1, S2)
    # the FP32 record rounds each velocity once, an error on the scale of C(0)
    # (the lags near a zero crossing of C have no relative accuracy to keep)
    np.testing.assert_allclose(C1, Co, rtol=0, atol=1e-6 * Co[0])


def test_record_capacity_and_end(M, water648):
    e = M.Engine(precision=M.MD_MIXED, seed=4)
    e.set_system(0, water648, **PARAMS)
    e.vacf_start(10)
    e.baoab(25)
    C, S, T = e.vacf(30)
    assert T == 10 and C[0] > 0 and (C[10:] == 0).all()
    # C(0) is the mean of sum m v^2 = 2 KE over the samples: about 3 n kB T
    kT = 0.0019872041 * 418.4 * 300.0
    assert 0.3 < C[0] / (3 * water648.n * kT) < 4.0
    e.vacf_start(0)
    C, S, T = e.vacf(30)
    assert T == 0 and (C == 0).all()


def test_vacf_of_each_replica(M, oracle_mod, water648):
    """two replicas in one context: each replica's VACF is its own (FP64,
    against the oracle's record of that replica's run)"""
    from test_gpu_ewald import perturbed
    w2 = perturbed(water648, seed=5)
    e = M.Engine(precision=M.MD_FP64, seed=6, max_replicas=2)
    e.set_system(0, water648, **PARAMS)
    e.set_system(1, w2, **PARAMS)
    e.vacf_start(40)
    e.baoab(40)
    for r, s in enumerate((water648, w2)):
        o = oracle_mod.Oracle(s, seed=6, replica=r, **PARAMS)
        o.vrec_enable(40)
        o.baoab(40)
        C, _, T = e.vacf(20, replica=r)
        assert T == 40
        np.testing.assert_allclose(C, oracle_mod.vacf(o.vrec(), s.mass, 20), rtol=1e-6)
