"""The pins must reject a broken oracle.

Each case plants one plausible mistake (a dropped term, a wrong sign, a
wrong index, a swapped operand) in a copy of the oracle's C source, builds it
on the CPU, and runs the pin suite against it in a subprocess: at least one
pin has to fail. The real oracle is never modified.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "koma_oracle.c")

MUTANTS = {
    "precession_sign": ("const double phi = -ORACLE_GAMMA * integral - dwj * dt;",
                        "const double phi = ORACLE_GAMMA * integral - dwj * dt;"),
    "no_trapezoid": ("0.5 * (J->gx[n] + J->gx[n + 1])", "J->gx[n]"),
    "drop_beta2_term": ("                                         - beta * beta * conj(mxy);", ";"),
    "alpha_not_conjugated": ("+ conj(alpha) * conj(alpha) * mxy", "+ alpha * alpha * mxy"),
    "mz_cross_term_sign": ("- 2.0 * creal(alpha * beta * conj(mxy));",
                           "+ 2.0 * creal(alpha * beta * conj(mxy));"),
    "t1_t2_swapped": ("const double e2 = exp(-dt / T2);", "const double e2 = exp(-dt / T1);"),
    "recovery_dropped": ("mz = mz * e1 + m0 * (1.0 - e1);", "mz = mz * e1;"),
    "adc_index": ("if (J->adc[n + 1]) {", "if (J->adc[n]) {"),
    "offresonance_dropped": ("const double phi = -ORACLE_GAMMA * integral - dwj * dt;",
                             "const double phi = -ORACLE_GAMMA * integral;"),
    "offresonance_dropped_in_rf": ("+ gzm * zm + dwj / ORACLE_GAMMA;", "+ gzm * zm;"),
    "full_angle": ("cos(phi / 2.0) - I * nz * sin(phi / 2.0)", "cos(phi) - I * nz * sin(phi)"),
    "nz_sign": ("cos(phi / 2.0) - I * nz * sin(phi / 2.0)", "cos(phi / 2.0) + I * nz * sin(phi / 2.0)"),
    "xy_swapped": ("const double fm = gxm * xm + gym * ym + gzm * zm;",
                   "const double fm = gxm * xm + gym * xm + gzm * zm;"),
    # motion x(t) = x + v t
    "motion_start_of_step": ("const double tm = t + 0.5 * dt;", "const double tm = t;"),
    "velocity_sign": ("const double xm = xj + vxj * tm", "const double xm = xj - vxj * tm"),
    "clock_not_advanced": ("        t += dt;\n", "\n"),
    "trapezoid_for_moving_spins": ("const double integral = dt / 6.0 * (f0 + 4.0 * fm + f1);",
                                   "const double integral = 0.5 * dt * (f0 + f1);"),
    "end_point_velocity_axis": ("J->gy[n + 1] * (yj + vyj * t1s)", "J->gy[n + 1] * (yj + vxj * t1s)"),
    "b1_conjugated": ("const double complex nxy = b1 / bnorm;", "const double complex nxy = conj(b1) / bnorm;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor not found: {old!r}"
    mutated = src.replace(old, new, 1)
    c_file = tmp_path / "mutant.c"
    c_file.write_text(mutated)
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                           "-ffp-contract=off", "-o", str(so), str(c_file), "-lm"])
    env = dict(os.environ, KOMA_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
