"""Mutation check of the oracle's pins.

Each case plants one plausible mistake in a copy of ``oracle/sd_oracle.c`` --
a dropped term, a wrong coefficient, sign, power or index, a wrong branch
threshold -- builds it with gcc, and runs ``tests/test_oracle_pins.py``
against that build (``SD_ORACLE_LIB``).  The pins must fail for every mutant:
a mutant that survives marks arithmetic that no independent fact checks.

Edits that leave the mathematics unchanged are not mutants here: T(r) is even
in r and symmetric, so swapping i and j in the separation, or the two indices
of a pair block, is not a mistake.
"""
import concurrent.futures
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "sd_oracle.c")

# (name, text in sd_oracle.c, replacement); the text must occur exactly once.
MUTANTS = [
    # Stokes self mobility 1/(6 pi eta a)
    ("mu0_constant", "1.0 / (6.0 * SDO_PI * eta * a)", "1.0 / (8.0 * SDO_PI * eta * a)"),
    # Oseen tensor (I + rr)/(8 pi eta r)
    ("oseen_sign", "t = (I + ee) / (8.0 * SDO_PI * eta * rn);", "t = (I - ee) / (8.0 * SDO_PI * eta * rn);"),
    ("oseen_power", "t = (I + ee) / (8.0 * SDO_PI * eta * rn);", "t = (I + ee) / (8.0 * SDO_PI * eta * rr2);"),
    ("oseen_constant", "t = (I + ee) / (8.0 * SDO_PI * eta * rn);", "t = (I + ee) / (6.0 * SDO_PI * eta * rn);"),
    # Rotne-Prager, far branch
    ("rp_first_sign", "(3.0 * a / (4.0 * rn)) * (I + ee)", "(3.0 * a / (4.0 * rn)) * (I - ee)"),
    ("rp_first_coef", "(3.0 * a / (4.0 * rn)) * (I + ee)", "(3.0 * a / (8.0 * rn)) * (I + ee)"),
    ("rp_second_sign", "(I - 3.0 * ee);", "(I + 3.0 * ee);"),
    ("rp_second_coef", "(a * a * a / (2.0 * rn * rn * rn)) * (I - 3.0 * ee)",
     "(a * a * a / (3.0 * rn * rn * rn)) * (I - 3.0 * ee)"),
    ("rp_second_dropped", "+ mu0 * (a * a * a / (2.0 * rn * rn * rn)) * (I - 3.0 * ee);", "+ 0.0;"),
    ("rp_second_power", "(a * a * a / (2.0 * rn * rn * rn)) * (I - 3.0 * ee)",
     "(a * a * a / (2.0 * rn * rn)) * (I - 3.0 * ee)"),
    # Yamakawa continuation r < 2a
    ("rpy_inner_diag", "(1.0 - 9.0 * rn / (32.0 * a)) * I", "(1.0 - 9.0 * rn / (16.0 * a)) * I"),
    ("rpy_inner_rr", "(3.0 * rn / (32.0 * a)) * ee", "(3.0 * rn / (16.0 * a)) * ee"),
    ("rpy_threshold", "} else if (tensor == SDO_RPY && rn < 2.0 * a) {\n                /* Yamakawa",
     "} else if (tensor == SDO_RPY && rn < 1.5 * a) {\n                /* Yamakawa"),
    ("rpy_inner_as_oseen", "} else if (tensor == SDO_RPY && rn < 2.0 * a) {\n                /* Yamakawa",
     "} else if (tensor == SDO_RP && rn < 2.0 * a) {\n                /* Yamakawa"),
    # mobility sum
    ("self_term_dropped", "acc[d] += mu0 * F[3 * i + d];", "acc[d] += 0.0 * F[3 * i + d];"),
    ("sum_wrong_force_index", "T[3 * al + 2] * F[3 * j + 2];", "T[3 * al + 2] * F[3 * i + 2];"),
    ("sum_wrong_component", "T[3 * al + 1] * F[3 * j + 1] +", "T[3 * al + 1] * F[3 * j + 2] +"),
    ("sum_uses_row_not_column", "T[3 * al] * F[3 * j] + T[3 * al + 1]", "T[3 * al] * F[3 * j] + T[3 * al]"),
    ("sum_skips_last_particle", "for (int j = 0; j < n; ++j) {\n        if (j == i) {",
     "for (int j = 0; j < n - 1; ++j) {\n        if (j == i) {"),
    ("assemble_self_block", "T[k] = (k % 4 == 0) ? mu0 : 0.0;", "T[k] = (k % 3 == 0) ? mu0 : 0.0;"),
    ("min_image_floor", "r[d] -= box[d] * nearbyint(r[d] / box[d]);", "r[d] -= box[d] * floor(r[d] / box[d]);"),
    # forces and Euler step
    ("gravity_dropped", "double f[3] = {g[0], g[1], g[2]};", "double f[3] = {0.0, 0.0, 0.0};"),
    ("repulsion_power", "pow(rn, 14.0)", "pow(rn, 13.0)"),
    ("repulsion_attractive", "f[d] += c * r[d];", "f[d] -= c * r[d];"),
    ("repulsion_cutoff_ignored", "if (rn < rep_rc) {", "if (rn < 1e300) {"),
    ("euler_half_step", "x[k] += dt * v[k];", "x[k] += 0.5 * dt * v[k];"),
    # derivatives
    ("profile_oseen_B", "*B = 3.0 * a / (4.0 * rn * rn * rn);", "*B = 3.0 * a / (4.0 * rn * rn);"),
    ("profile_inner_dA", "*dA = -9.0 / (32.0 * a);", "*dA = 9.0 / (32.0 * a);"),
    ("profile_inner_dB", "*dB = -3.0 / (32.0 * a * rn * rn);", "*dB = -3.0 / (16.0 * a * rn * rn);"),
    ("profile_far_dA", "- 3.0 * a3 / (2.0 * pow(rn, 4));", "- 3.0 * a3 / (4.0 * pow(rn, 4));"),
    ("profile_far_dB", "+ 15.0 * a3 / (2.0 * pow(rn, 6));", "+ 15.0 * a3 / (4.0 * pow(rn, 6));"),
    ("dtensor_term_dropped", "B * (d_ag * r[be] + r[al] * d_bg)", "B * (d_ag * r[be])"),
    ("vjp_reciprocal_dropped", "+ w[3 * j + al] * dT[9 * g + 3 * al + be] * F[3 * k + be];", ";"),
    ("vjp_gF_uses_F", "if (gF) st = sdo_mobility_apply(tensor, a, eta, box, n, x, w, gF, nthreads);",
     "if (gF) st = sdo_mobility_apply(tensor, a, eta, box, n, x, F, gF, nthreads);"),
    ("adjoint_gF_no_dt", "gF[k] += dt * tF[k];", "gF[k] += tF[k];"),
    ("adjoint_lambda_sign", "lam[k] += dt * tx[k];", "lam[k] -= dt * tx[k];"),
    ("adjoint_wrong_state", "const double *xs = traj + (size_t)s * m;\n        st = sdo_vjp",
     "const double *xs = traj + (size_t)(s + 1) * m;\n        st = sdo_vjp"),
    ("adjoint_gravity_dropped", "F[k] = (fext ? fext[k] : 0.0) + g[k % 3];", "F[k] = (fext ? fext[k] : 0.0);"),
    # lubrication (Sec. 2.3) and its use in the Euler step
    ("lub_reynolds_coef", "1.0 / (4.0 * sg)", "1.0 / (2.0 * sg)"),
    ("lub_normal_log_coef", "(9.0 / 40.0) * log(sg)", "(9.0 / 20.0) * log(sg)"),
    ("lub_tangential_coef", "-(1.0 / 6.0) * log(sg)", "-(1.0 / 3.0) * log(sg)"),
    ("lub_tangential_dropped", "(normal * ee + tangential * (I - ee))", "(normal * ee)"),
    ("lub_projector_swapped", "(normal * ee + tangential * (I - ee))", "(normal * (I - ee) + tangential * ee)"),
    ("lub_sign", "f[al] -= zv / mu0;", "f[al] += zv / mu0;"),
    ("lub_times_mu0", "f[al] -= zv / mu0;", "f[al] -= zv * mu0;"),
    ("lub_cutoff", "sg > 0.0 && sg < 1.0", "sg > 0.0 && sg < 2.0"),
    ("lub_overlap_kept", "sg > 0.0 && sg < 1.0", "sg > -1.0 && sg < 1.0"),
    ("lub_own_velocity_only", "v[3 * i] - v[3 * j], v[3 * i + 1] - v[3 * j + 1], v[3 * i + 2] - v[3 * j + 2]",
     "v[3 * i], v[3 * i + 1], v[3 * i + 2]"),
    ("euler_lub_not_applied", "if (lub) sdo_lubrication(a, eta, box, n, x, v, F);", ""),
]


def _run_mutant(name, old, new, workdir):
    src = open(SRC).read()
    assert src.count(old) == 1, (name, src.count(old))
    path = os.path.join(workdir, name + ".c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    lib = os.path.join(workdir, "lib_" + name + ".so")
    subprocess.check_call(["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fPIC", "-shared", "-std=c99",
                           path, "-o", lib, "-lm"])
    env = dict(os.environ, SD_ORACLE_LIB=lib, OMP_NUM_THREADS="1")
    p = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        "-x", "-q", "-m", "not gpu", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    failed = [l for l in p.stdout.splitlines() if l.startswith("FAILED") or l.startswith("ERROR")]
    return name, p.returncode, failed


def test_mutant_sources_apply_once():
    src = open(SRC).read()
    for name, old, _ in MUTANTS:
        assert src.count(old) == 1, name


def test_pins_kill_every_mutant(orc, tmp_path):
    workers = max(1, min(len(MUTANTS), os.cpu_count() or 1))
    with concurrent.futures.ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(lambda m: _run_mutant(m[0], m[1], m[2], str(tmp_path)), MUTANTS))
    survivors = [name for name, rc, _ in results if rc == 0]
    assert not survivors, "mutants the pins do not catch: %s" % survivors
    for name, rc, _ in results:
        assert rc == 1, (name, rc)   # a test failure, not a crash of the run
