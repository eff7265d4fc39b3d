"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake (a dropped term, a flipped sign, a wrong index or
coefficient) in a copy of the oracle's C source, builds it, and runs the pin
tests against that copy in a subprocess: every run must fail.  The mistakes
are planted in the oracle, on the CPU; nothing here touches a GPU.
"""
import os
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "nbody_oracle.c")
PINS = ["tests/test_oracle_force.py", "tests/test_oracle_hermite.py", "tests/test_oracle_adjoint.py"]
# mistakes in the summation variants only touch that code: their own pins suffice
SUMMATION_PINS = ["tests/test_oracle_summation.py"]
SUMMATION_PREFIXES = ("pair32_", "fixed_", "sorted_", "integrator_ignores_summation")

MUTATIONS = {
    "force_sign_repulsive": ("dx[c] = x[3 * j + c] - x[3 * i + c];", "dx[c] = x[3 * i + c] - x[3 * j + c];"),
    "jerk_drop_factor_3": ("3.0 * xv * dx[c] / r5", "xv * dx[c] / r5"),
    "jerk_wrong_sign": ("dv[c] / r3 - 3.0", "dv[c] / r3 + 3.0"),
    "jerk_dv_transposed": ("dv[c] = v[3 * j + c] - v[3 * i + c];", "dv[c] = v[3 * i + c] - v[3 * j + c];"),
    "force_no_softening": ("dx[2] * dx[2] + eps * eps;", "dx[2] * dx[2];"),
    "force_mass_index": ("ai[c] += m[j] * dx[c] / r3;", "ai[c] += m[i] * dx[c] / r3;"),
    "force_self_term_kept": ("if (j == i) continue;\n            double dx[3], dv[3];", "double dx[3], dv[3];"),
    "pot_wrong_power": ("pi -= m[j] / r;", "pi -= m[j] / r2;"),
    "predict_dt_over_2": ("(a[c] + (dt / 3.0) * k[c])", "(a[c] + (dt / 2.0) * k[c])"),
    "predict_v_drop_jerk": ("vp[c] = v[c] + (a[c] + (dt / 2.0) * k[c]) * dt;", "vp[c] = v[c] + a[c] * dt;"),
    "corrector_a2_swapped": ("- (2.0 * k[c] + kp[c]) * dt", "- (k[c] + 2.0 * kp[c]) * dt"),
    "corrector_a3_coeff": ("a3[c] / 20.0", "a3[c] / 24.0"),
    "corrector_v_coeff": ("a3[c] / 4.0", "a3[c] / 6.0"),
    "aarseth_swapped_term": ("double num = na * ns + nk * nk;", "double num = na * ns + na * na;"),
    "aarseth_crackle_power": ("cr[c] = 6.0 * a3[c] / dt3;", "cr[c] = 6.0 * a3[c] / dt2;"),
    "level_off_by_one": ("k = 1 - e;", "k = -e;"),
    "doubling_not_commensurate": ("if (t_new % twice_old == 0) return k_old - 1;", "return k_old - 1;"),
    "block_only_first_particle": ("== tn) act[na++] = (int32_t)i;", "== tn) { act[na++] = (int32_t)i; break; }"),
    "block_end_time_off_by_one": ("int64_t e = t[i] + ((int64_t)1 << (ORC_TICK_BITS - lev[i]));",
                                  "int64_t e = t[i] + ((int64_t)1 << (ORC_TICK_BITS - lev[i] - 1));"),
    "energy_kinetic_no_half": ("t += 0.5 * m[i] *", "t += m[i] *"),
    "energy_no_softening": ("d2 * d2 + eps * eps);", "d2 * d2);"),
    "vjp_drop_15_term": ("\n                                    + 15.0 * s * kd * d[c] / r7);", ");"),
    "vjp_gw_wrong_sign": ("vbar[3 * j + c] += gw;\n                vbar[3 * i + c] -= gw;",
                          "vbar[3 * j + c] -= gw;\n                vbar[3 * i + c] += gw;"),
    "vjp_mass_missing_term": ("mbar[j] += ad / r3 + kw / r3 - 3.0 * s * kd / r5;",
                              "mbar[j] += ad / r3 - 3.0 * s * kd / r5;"),
    "traj_predictor_transpose": ("kb[c] += xpb * q * h * dt + vpb * h * dt;", "kb[c] += xpb * h * dt + vpb * h * dt;"),
    "traj_corrector_coeff": ("double a3b = xbar[c] * dt * dt / 20.0", "double a3b = xbar[c] * dt * dt / 12.0"),
    "traj_k1b_sign": ("k1b[c] = kb[c] + a3b * dt - a2b * dt;", "k1b[c] = kb[c] + a3b * dt + a2b * dt;"),
    "traj_no_initial_force_vjp": ("        xbar[c] += xg[c];\n        vbar[c] += vg[c];\n", ""),
    "pair32_lo_dropped": ("dx[c] = (pj->hi[c] - pi->hi[c]) + (pj->lo[c] - pi->lo[c]);",
                          "dx[c] = pj->hi[c] - pi->hi[c];"),
    "pair32_jerk_sign": ("t[3 + c] = fk * (u[c] + b * dx[c]);", "t[3 + c] = fk * (u[c] - b * dx[c]);"),
    "pair32_b_coeff": ("float b = (-3.0f * rv) * rinv2;", "float b = (-2.0f * rv) * rinv2;"),
    "pair32_no_softening": ("float r2 = d2 + eps2;", "float r2 = d2;"),
    "pair32_key_softened_inverse_square": ("*key = fminf(mr3 * sqrtf(d2), FLT_MAX);",
                                           "*key = fminf(mr * rinv, FLT_MAX);"),
    "fixed_truncates": ("Y[q] += (__int128)llrintf(t[q]);", "Y[q] += (__int128)(long long)t[q];"),
    "fixed_scale_off_by_one": ("s[q] = 56 - e[q];", "s[q] = 57 - e[q];"),
    "fixed_jerk_floor_truncated": ("3 + Em + Ev - orc_floor_half(3 * F)", "3 + Em + Ev - (3 * F) / 2"),
    "fixed_conversion_drops_sign": ("return neg ? -d : d;", "return d;"),
    "fixed_pot_uses_jerk_scale": ("ldexp(1.0, -s[q < 3 ? 0 : (q < 6 ? 1 : 2)])", "ldexp(1.0, -s[q < 3 ? 0 : 1])"),
    "sorted_descending": ("if (a->key != b->key) return a->key < b->key ? -1 : 1;",
                          "if (a->key != b->key) return a->key > b->key ? -1 : 1;"),
    "sorted_ties_reversed": ("return a->j < b->j ? -1 : (a->j > b->j);", "return a->j > b->j ? -1 : (a->j < b->j);"),
    "integrator_ignores_summation": ("if (mode == ORC_SUM_FP64) {\n        orc_force(",
                                     "if (1) {\n        orc_force("),
}


def _run(name, tmpdir):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    path = os.path.join(tmpdir, name + ".c")
    lib = os.path.join(tmpdir, name + ".so")
    open(path, "w").write(src.replace(old, new))
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
                    "-shared", "-o", lib, path, "-lm"], check=True)
    env = dict(os.environ, NBODY_ORACLE_LIB=lib, OMP_NUM_THREADS="1")
    pins = SUMMATION_PINS if name.startswith(SUMMATION_PREFIXES) else PINS
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *pins],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode


@pytest.mark.slow
def test_every_planted_mistake_is_caught():
    names = sorted(MUTATIONS)
    with tempfile.TemporaryDirectory() as d:
        with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
            codes = dict(zip(names, ex.map(lambda n: _run(n, d), names)))
    survived = [n for n, c in codes.items() if c == 0]
    assert not survived, "mutations not caught by the pins: %s" % survived
    assert all(c == 1 for c in codes.values()), codes  # failed tests, not crashes
