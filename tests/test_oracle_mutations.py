"""The oracle's pins catch plausible mistakes. Each case writes oracle.c
with one planted mistake (a dropped term, a wrong sign or factor, a wrong
index rule) into a temporary folder, compiles it there, and runs the pin
that should catch it in a child pytest against that library (through
ORACLE_MUTANT_LIB): the pin must fail. A control run of the same machinery
on the unedited source must pass. Nothing here touches oracle/ itself."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")
CHAIN = "tests/test_oracle_dynamics.py::test_multiple_time_step_jumps_sample_boltzmann_harmonic_chain"

# (name, text in oracle.c, replacement, pin to run)
MUTANTS = [
    ("Philox with nine rounds",
     "for (int r = 0; r < 10; ++r)", "for (int r = 0; r < 9; ++r)",
     "tests/test_oracle_primitives.py::test_philox_known_answers"),
    ("Theta with 0.9 phi",
     "double t = eta * nPhi(eta) + nphi(eta);", "double t = eta * nPhi(eta) + 0.9 * nphi(eta);",
     "tests/test_oracle_primitives.py::test_theta_identities"),
    ("G~ mixture weight eta / (eta + 1)",
     "double pg = eta / (eta + 1.0 / sqrt(2.0 * OR_PI));", "double pg = eta / (eta + 1.0);",
     "tests/test_oracle_primitives.py::test_gtilde_law"),
    ("switch slope with the wrong sign",
     "return -30.0 * t * t * (1.0 - t) * (1.0 - t) / s->p.h_switch;",
     "return 30.0 * t * t * (1.0 - t) * (1.0 - t) / s->p.h_switch;",
     "tests/test_oracle_primitives.py::test_pair_derivative_is_gradient_of_energy"),
    ("DSF without its value shift",
     "return erfc(a * r) / r - eR + fR * (r - R);", "return erfc(a * r) / r + fR * (r - R);",
     "tests/test_oracle_primitives.py::test_dsf_closed_form"),
    ("angle gradient on an end atom with the wrong sign",
     "double ga = (cth * a[c] / ra - b[c] / rb) / (ra * sth);",
     "double ga = (b[c] / rb - cth * a[c] / ra) / (ra * sth);",
     "tests/test_oracle_primitives.py::test_total_gradient_finite_differences"),
    ("intramolecular pairs kept in the nonbonded sum",
     "if (r2 >= R2 || excluded(s, i, j)) continue;", "if (r2 >= R2) continue;",
     "tests/test_oracle_primitives.py::test_single_molecule_has_no_nonbonded_terms"),
    ("uncharged partners kept in the rings",
     "if (kind >= s->nr || sw >= R || s->q[i] * s->q[j] == 0.0) return 0;",
     "if (kind >= s->nr || sw >= R) return 0;",
     "tests/test_oracle_primitives.py::test_jump_lists_definition"),
    ("ring of a proposal always ring 0",
     "if (target < cum) { Y = y; break; }", "if (target < cum) { Y = 0; break; }",
     "tests/test_oracle_dynamics.py::test_cprime_first_jump_survival_a0"),
    ("speed bound without its s^2 |a|^2 term",
     "double B = sqrt(vv + sr * sr * aa + 2.0 * sr * (va > 0.0 ? va : 0.0));",
     "double B = sqrt(vv + 2.0 * sr * (va > 0.0 ? va : 0.0));",
     "tests/test_oracle_dynamics.py::test_cprime_first_jump_survival_with_drift"),
    ("BPS reflection factor 1 instead of 2",
     "for (int c = 0; c < 3; ++c) v[c] -= 2.0 * vg / gg * g[c];",
     "for (int c = 0; c < 3; ++c) v[c] -= 1.0 * vg / gg * g[c];",
     "tests/test_oracle_dynamics.py::test_jprime_single_bounce_law"),
    ("O-step noise amplitude without its square root",
     "double c2 = sqrt(one_m / (s->beta * s->mt[i]));", "double c2 = one_m / sqrt(s->beta * s->mt[i]);",
     "tests/test_oracle_dynamics.py::test_baoab_exact_harmonic_configurations"),
    ("list rebuild threshold at 2.5 skins",
     "li = 0.5 * s->p.skin;", "li = 2.5 * s->p.skin;",
     "tests/test_oracle_dynamics.py::test_lists_cover_the_current_shells_during_dynamics"),
    ("BAOAB-RESPA outer kick 0.6 D",
     "        kick(s, s->al, 0.5 * D);\n        for (int k = 0; k < n_inner; ++k) inner_bonded(s, dt, k < n_inner - 1);",
     "        kick(s, s->al, 0.6 * D);\n        for (int k = 0; k < n_inner; ++k) inner_bonded(s, dt, k < n_inner - 1);",
     "tests/test_oracle_dynamics.py::test_multiple_time_step_energy_error_second_order"),
    ("Ewald self term with the wrong sign",
     "e -= OR_COULOMB * a / sqrt(OR_PI) * s->q[i] * s->q[i];",
     "e += OR_COULOMB * a / sqrt(OR_PI) * s->q[i] * s->q[i];",
     "tests/test_oracle_ewald.py::test_total_ewald_energy_does_not_depend_on_alpha"),
    ("PME influence function without |b(m)|^-2",
     "/ msq * bmod[m0] * bmod[m1] * bmod[m2];", "/ msq;",
     "tests/test_oracle_ewald.py::test_smooth_pme_matches_the_plain_sum"),
    ("JUMP-RESPA1 closing slow kick with a stale force",
     "        if (ew) { accel(s, 6, s->al); kick(s, s->al, 0.5 * D); }",
     "        if (ew) { kick(s, s->al, 0.5 * D); }",
     "tests/test_oracle_ewald.py::test_jump_mts_equals_baoab_mts_under_ewald_without_jump_range"),
    ("JUMP-RESPA jumps over the inner half step",
     "cphase(s, s->as, 0.5 * D, s0", "cphase(s, s->as, 0.5 * dt, s0",
     CHAIN + "[jump_respa-0]"),
    ("JUMP-RESPA C' drift that still holds the bonded force",
     "accel(s, 3, s->as);\n        jphase(s, 0.5 * D, s0, 1);",
     "accel(s, 5, s->as);\n        jphase(s, 0.5 * D, s0, 1);",
     CHAIN + "[jump_respa-0]"),
    ("JUMP-RESPA LJ bounces over the inner half step",
     "jphase(s, 0.5 * D, s0", "jphase(s, 0.5 * dt, s0",
     CHAIN + "[jump_respa-0]"),
    ("JUMP-RESPA1 jumps over the outer half step",
     "cphase(s, s->as, 0.5 * kap, s0", "cphase(s, s->as, 0.5 * D, s0",
     CHAIN + "[jump_respa1-0]"),
    ("JUMP-RESPA1 C' drift that still holds the bonded force",
     "accel(s, 3, s->as);\n            jphase(s, 0.5 * kap, s0, 1);",
     "accel(s, 5, s->as);\n            jphase(s, 0.5 * kap, s0, 1);",
     CHAIN + "[jump_respa1-0]"),
    ("JUMP-RESPA1 opening slow kick over the mid half step",
     "        if (ew) kick(s, s->al, 0.5 * D);\n        for (int j = 0; j < n_outer; ++j) {",
     "        if (ew) kick(s, s->al, 0.5 * kap);\n        for (int j = 0; j < n_outer; ++j) {",
     CHAIN + "[jump_respa1-2]"),
    ("Ewald exclusion correction with the wrong sign",
     "if (j > i) e -= qq * erf(a * r) / r;", "if (j > i) e += qq * erf(a * r) / r;",
     "tests/test_oracle_ewald.py::test_total_ewald_energy_does_not_depend_on_alpha"),
    ("Ewald real-space derivative with half its Gaussian term",
     "return -(erfc(a * r) / r + 2.0 * a / sqrt(OR_PI) * exp(-a * a * r * r)) / r;",
     "return -(erfc(a * r) / r + 1.0 * a / sqrt(OR_PI) * exp(-a * a * r * r)) / r;",
     "tests/test_oracle_ewald.py::test_total_ewald_gradient_is_the_derivative_of_its_energy"),
    ("C' acceptance with sqrt(beta m) for sqrt(beta / m)",
     "p = sqrt(beta / mt) * or_theta(eta) / eps0 / LamY[Y];", "p = sqrt(beta * mt) * or_theta(eta) / eps0 / LamY[Y];",
     "tests/test_oracle_dynamics.py::test_cprime_first_jump_survival_a0"),
    ("C' jump kernel without the eps^2 of its normalisation",
     "double coef = 2.0 * eps / (sqrt(beta * mt) * (1.0 + eps * eps)) * (eta + Gt) / gn;",
     "double coef = 2.0 * eps / (sqrt(beta * mt) * (1.0 + eps)) * (eta + Gt) / gn;",
     "tests/test_oracle_dynamics.py::test_jump_samples_boltzmann_two_body"),
    ("JUMP's closing C' with the opening step's force",
     "        maybe_rebuild(s);\n        accel(s, 5, s->a0);\n        jphase(s, 0.5 * tau, s0, 1);",
     "        maybe_rebuild(s);\n        jphase(s, 0.5 * tau, s0, 1);",
     "tests/test_oracle_dynamics.py::test_jump_samples_boltzmann_two_body"),
    ("BAOAB-RESPA1 closing mid-level kick 0.6 kappa",
     "            accel(s, 3, s->as);\n            kick(s, s->as, 0.5 * kap);\n            if (j < n_outer - 1) vrec(s);",
     "            accel(s, 3, s->as);\n            kick(s, s->as, 0.6 * kap);\n            if (j < n_outer - 1) vrec(s);",
     "tests/test_oracle_dynamics.py::test_multiple_time_step_energy_error_second_order"),
    ("BJAOAJB jumps with the drift of F0",
     "        cphase(s, zero, 0.5 * tau, s0, 0);", "        cphase(s, s->a0, 0.5 * tau, s0, 0);",
     "tests/test_oracle_dynamics.py::test_bjaoajb_is_baoab_without_jumps_and_keeps_temperature"),
    ("BAOAB velocity recorded before the closing kick",
     "        kick(s, s->a0, 0.5 * tau);\n        s->step++;\n        vrec(s);\n    }\n    check_finite(s);\n"
     "    return (int)s->err;\n}\n\n/* JUMP: C'",
     "        vrec(s);\n        kick(s, s->a0, 0.5 * tau);\n        s->step++;\n    }\n    check_finite(s);\n"
     "    return (int)s->err;\n}\n\n/* JUMP: C'",
     "tests/test_oracle_vacf.py::test_record_places_follow_the_integrator_identities"),
    ("VACF normalised by T instead of T - k",
     "acc /= (double)(T - k);", "acc /= (double)(T);",
     "tests/test_oracle_vacf.py::test_vacf_of_a_cosine_matches_its_closed_form"),
]


def build_variant(tmp_path, text):
    import oracle
    src = tmp_path / "oracle.c"
    src.write_text(text)
    (tmp_path / "oracle.h").write_text(open(os.path.join(ROOT, "oracle", "oracle.h")).read())
    lib = tmp_path / "liboracle_mutant.so"
    subprocess.run(["gcc", *oracle.CFLAGS, "-o", str(lib), str(src), "-lm"], check=True)
    return str(lib)


def run_pins(lib, pins):
    env = dict(os.environ, ORACLE_MUTANT_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *pins],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return r.returncode, (r.stdout.strip().splitlines() or [""])[-1]


@pytest.mark.slow
def test_control_unedited_oracle_passes_the_pins(tmp_path):
    """the same build and child run on the unedited source pass every pin used below"""
    lib = build_variant(tmp_path, open(SRC).read())
    rc, tail = run_pins(lib, sorted({m[3] for m in MUTANTS}))
    assert rc == 0 and " passed" in tail and "failed" not in tail, tail


@pytest.mark.slow
@pytest.mark.parametrize("name,old,new,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_its_pin(tmp_path, name, old, new, pin):
    text = open(SRC).read()
    assert text.count(old) >= 1, f"site of '{name}' not found in oracle.c"
    lib = build_variant(tmp_path, text.replace(old, new))
    rc, tail = run_pins(lib, [pin])
    # a test failure, not a collection or build error
    assert rc != 0 and " failed" in tail, f"'{name}' against {pin}: {tail}"
