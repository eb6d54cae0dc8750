"""Planted mistakes in the oracle: every one must fail a pin.

Each case copies the oracle's C sources (oracle/olbm_oracle.c, oracle/olbm_core.inc)
to a temporary folder, plants one plausible mistake (a dropped term, a wrong sign,
a wrong index or axis, a transposed operand, a mixed-up velocity table), compiles
the copy with the oracle's own flags and runs the CPU pins (tests/test_oracle_pins.py
and tests/test_golden_cpu.py) against it in a subprocess (OLBM_ORACLE_LIB points the
oracle's loader at the copy). The pins must fail for every mutant, and must pass
for the unmodified copy built the same way. The oracle itself is never modified.
The exact isothermal Riemann solution (oracle/riemann.py) gets the same treatment
against tests/test_riemann_cpu.py, loaded in place of the original in a subprocess.

Left out because it is not a mistake: dropping the trace term -C_i^2/D delta_ab on
the i side of Eq. 2's contraction. The k-sum it multiplies is traceless, so that
term contributes C_i^2/2 (T_xx + T_yy) = 0 and the mutant computes the same values.
The trace term on the k side is planted (oreg_dropped_trace_k) and caught.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")
PINS = [os.path.join("tests", "test_oracle_pins.py"), os.path.join("tests", "test_golden_cpu.py")]
CORE, MAIN = "olbm_core.inc", "olbm_oracle.c"

# (name, passage, [(file, text in the oracle, planted text), ...])
MUTANTS = [
    ("geq_sign_of_cu", "Eq. 10",
     [(CORE, "(double)c2 - 1.0 + (double)c * u + u * u + theta", "(double)c2 - 1.0 - (double)c * u + u * u + theta")]),
    ("geq_dropped_u2", "Eq. 10",
     [(CORE, "(double)c2 - 1.0 + (double)c * u + u * u + theta", "(double)c2 - 1.0 + (double)c * u + theta")]),
    ("geq_normalisation", "Eq. 10",
     [(CORE, "(1.0 - 2.0 * (double)c2) / (double)(1 << c2)", "(1.0 - 2.0 * (double)c2) / 2.0")]),
    ("heq_dropped_theta", "Sec. 5.1, second LBGK reading",
     [(CORE, "(cu * cu - theta * usq)", "(cu * cu - usq)")]),
    ("heq_rest_weight", "Sec. 5.1, second LBGK reading",
     [(CORE, "const double wx = CX[i] == 0 ? 1.0 - theta : 0.5 * theta;",
       "const double wx = CX[i] == 0 ? 1.0 - theta : theta;")]),
    ("moments_wrong_axis", "Sec. 1",
     [(CORE, "*uy = jy / r;", "*uy = jx / r;")]),
    ("oreg_transposed_index", "Eq. 2",
     [(CORE, "contraction = contraction + (Ci[a] * Ci[b] - Ci2 / D * dab) * ksum;",
       "contraction = contraction + (Ci[a] * Ci[a] - Ci2 / D * dab) * ksum;")]),
    ("oreg_dropped_trace_k", "Eq. 2",
     [(CORE, "ksum = ksum + ((double)(cka * ckb) - (double)ck2 / D * dab) * fneq[k];",
       "ksum = ksum + ((double)(cka * ckb)) * fneq[k];")]),
    ("oreg_f_for_fneq", "Eq. 2",
     [(CORE, "- (double)ck2 / D * dab) * fneq[k];", "- (double)ck2 / D * dab) * f[k];")]),
    ("oreg_prefactor", "Eq. 2",
     [(CORE, "feq[i] / (2.0 * rho * theta * theta) * contraction", "feq[i] / (rho * theta * theta) * contraction")]),
    ("psi_wrong_axis", "Eq. 6a",
     [(CORE, "py = py + (double)CY[i] * foreg[i];", "py = py + (double)CX[i] * foreg[i];")]),
    ("pref_sign", "Eq. 12",
     [(CORE, "return -1.0 / (4.0 * theta * theta) * s;", "return 1.0 / (4.0 * theta * theta) * s;")]),
    ("pref_sum_of_axes", "Eq. 12",
     [(CORE, "(double)(CX[i] * CX[i] - CY[i] * CY[i]) * g[i]", "(double)(CX[i] * CX[i] + CY[i] * CY[i]) * g[i]")]),
    ("pitilde_xx_sign", "Eq. 11b",
     [(CORE, "pit[0] = pref * (-(theta * (1.0 - 3.0 * theta)", "pit[0] = pref * ((theta * (1.0 - 3.0 * theta)")]),
    ("pitilde_yy_theta_term", "Eq. 11b",
     [(CORE, "pit[1] = pref * (theta * (1.0 - 3.0 * theta)", "pit[1] = pref * (theta * (1.0 - 2.0 * theta)")]),
    ("pitilde_xy_order", "Eq. 11b",
     [(CORE, "pit[2] = pref * (ux * uy * (ux * ux - uy * uy));", "pit[2] = pref * (ux * uy * (uy * uy - ux * ux));")]),
    ("partial_sign", "Eq. 14",
     [(CORE, "Psi[i] = -0.5 * ((double)CX[i] * psi[0]);", "Psi[i] = 0.5 * ((double)CX[i] * psi[0]);")]),
    ("partial_axis", "Eq. 14",
     [(CORE, "Psi[i] = -0.5 * ((double)CY[i] * psi[1]);", "Psi[i] = -0.5 * ((double)CY[i] * psi[0]);")]),
    ("complete_abar", "Eq. 15",
     [(CORE, "v = -2.0 * (pit[1] - (double)CX[i] * psi[0]);", "v = -2.0 * (pit[0] - (double)CX[i] * psi[0]);")]),
    ("complete_psi_sign", "Eq. 15",
     [(CORE, "v = -2.0 * (pit[0] - (double)CY[i] * psi[1]);", "v = -2.0 * (pit[0] + (double)CY[i] * psi[1]);")]),
    ("complete_dropped_cc_xy", "Eq. 15",
     [(CORE, "v = pit[0] + pit[1] + (double)(CX[i] * CY[i]) * pit[2];", "v = pit[0] + pit[1] + pit[2];")]),
    ("complete_scale", "Eq. 15",
     [(CORE, "Psi[i] = -0.25 * v;", "Psi[i] = -0.5 * v;")]),
    ("neq_variant_on_foreg", "Eq. 12, f^neq reading",
     [(CORE, "FN(pitilde)(FN(pref)(fneq, theta), ux, uy, theta, pit);",
       "FN(pitilde)(FN(pref)(g, theta), ux, uy, theta, pit);")]),
    ("relaxation_factor", "Eq. 1a",
     [(CORE, "const double omega_p = 1.0 - 1.0 / tau;", "const double omega_p = 1.0 / tau;")]),
    ("poly_lbgk_dispatch", "Eq. 1a, model 5",
     [(CORE, "if (model == 0 || model == 5) {", "if (model == 0) {")]),
    ("bounce_back_axis", "Sec. 5.2",
     [(CORE, "if (CX[j] == -CX[i] && CY[j] == -CY[i]) fs[i] = f[j];",
       "if (CX[j] == -CX[i] && CY[j] == CY[i]) fs[i] = f[j];")]),
    ("streaming_direction", "Eq. 1b",
     [(CORE, "const int xd = (x + CX[i] + nx) % nx;", "const int xd = (x - CX[i] + nx) % nx;")]),
    ("velocity_numbering", "Fig. 1a",
     [(MAIN, "static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};",
       "static const int CX[9] = {0, 1, 0, -1, 0, 1, 1, -1, -1};"),
      (MAIN, "static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};",
       "static const int CY[9] = {0, 0, 1, 0, -1, 1, -1, -1, 1};")]),
    ("diagnostics_energy_half", "diagnostics",
     [(MAIN, "nsum_add(&ke, 0.5 * (jx * jx + jy * jy) / rho);", "nsum_add(&ke, (jx * jx + jy * jy) / rho);")]),
    ("diagnostics_momentum_axis", "diagnostics",
     [(MAIN, "jy += (double)CY[i] * v;", "jy += (double)CX[i] * v;")]),
    ("run_result_left_in_scratch", "Eq. 1, odd step counts",
     [(MAIN, "  if (a != f) memcpy(f, a, n9 * sizeof(double));\n", "")]),
    ("moments_field_transposed_layout", "Sec. 1, [i][y][x] layout",
     [(MAIN, "    for (int i = 0; i < Q9; ++i) fl[i] = f[(size_t)i * N + n];\n    r_moments(fl, &rho[n], &ux[n], &uy[n]);",
       "    for (int i = 0; i < Q9; ++i) fl[i] = f[n * Q9 + (size_t)i];\n    r_moments(fl, &rho[n], &ux[n], &uy[n]);")]),
    ("complex_step_init_axes", "Eq. 10, complex-step twin",
     [(MAIN, "z_init((const double _Complex*)rho_ri, (const double _Complex*)ux_ri,\n         (const double _Complex*)uy_ri,",
       "z_init((const double _Complex*)rho_ri, (const double _Complex*)uy_ri,\n         (const double _Complex*)ux_ri,")]),
]


def _build(folder, edits):
    """Copy the oracle's C sources into `folder`, apply the edits, compile; returns the library."""
    os.makedirs(folder)
    for name in (CORE, MAIN):
        shutil.copy(os.path.join(ORACLE, name), os.path.join(folder, name))
    for fname, old, new in edits:
        path = os.path.join(folder, fname)
        text = open(path).read()
        assert text.count(old) == 1, f"{fname}: the text to replace must occur once: {old!r}"
        open(path, "w").write(text.replace(old, new))
    lib = os.path.join(folder, "liboracle.so")
    subprocess.run(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-o", lib,
                    os.path.join(folder, MAIN), "-lm"], check=True, capture_output=True, cwd=folder)
    return lib


def _pins(lib):
    """Run the CPU pins against the library; (exit status, last lines of the output)."""
    env = dict(os.environ, OLBM_ORACLE_LIB=lib, OMP_NUM_THREADS="2")
    res = subprocess.run([sys.executable, "-m", "pytest", *PINS, "-x", "-q", "-p", "no:cacheprovider",
                          "-m", "not gpu"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return res.returncode, "\n".join((res.stdout + res.stderr).splitlines()[-15:])


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    base = tmp_path_factory.mktemp("oracle_mutants")
    cases = [("unmodified", [])] + [(name, edits) for name, _, edits in MUTANTS]

    def one(case):
        name, edits = case
        return name, _pins(_build(str(base / name), edits))

    with ThreadPoolExecutor(max_workers=max(1, min(8, (os.cpu_count() or 2) // 2))) as pool:
        return dict(pool.map(one, cases))


def test_unmodified_copy_passes_the_pins(outcomes):
    status, tail = outcomes["unmodified"]
    assert status == 0, tail


@pytest.mark.parametrize("name,passage", [(m[0], m[1]) for m in MUTANTS])
def test_planted_mistake_fails_a_pin(outcomes, name, passage):
    status, tail = outcomes[name]
    # exit status 1: tests ran and one failed (not a collection or usage error)
    assert status == 1, f"{name} ({passage}) was not caught by the pins (status {status}):\n{tail}"


# The exact isothermal Riemann solution (oracle/riemann.py, the shocktube's checker of Sec. 5.2)
# against its pins (tests/test_riemann_cpu.py): (name, text in riemann.py, planted text).
RIEMANN_MUTANTS = [
    ("shock_curve_denominator", "return c * (rho - rho_k) / s,", "return c * (rho - rho_k) / rho,"),
    ("rarefaction_curve_sign", "return c * math.log(rho / rho_k), c / rho", "return c * math.log(rho_k / rho), c / rho"),
    ("middle_velocity_sign", "return rho, u_l - _wave_curve(rho, rho_l, c)[0]",
     "return rho, u_l + _wave_curve(rho, rho_l, c)[0]"),
    ("newton_velocity_jump_sign", "step = (fl + fr + u_r - u_l) / (dl + dr)", "step = (fl + fr - u_r + u_l) / (dl + dr)"),
    ("left_shock_speed", "sl = u_l - c * math.sqrt(rs / rho_l)", "sl = u_l - c * math.sqrt(rho_l / rs)"),
    ("right_shock_speed", "sr = u_r + c * math.sqrt(rs / rho_r)", "sr = u_r + c * math.sqrt(rho_r / rs)"),
    ("left_fan_head", "elif z < u_l - c:", "elif z < u_l:"),
    ("left_fan_invariant", "rho[k] = rho_l * math.exp((u_l - u[k]) / c)", "rho[k] = rho_l * math.exp((u[k] - u_l) / c)"),
    ("right_fan_characteristic", "u[k] = z - c", "u[k] = z + c"),
    ("l1_without_abs", "np.mean(np.abs(r - exact_rho))", "np.mean(r - exact_rho)"),
    ("tv_without_exact_profile", "np.abs(np.diff(r)).sum() - np.abs(np.diff(exact_rho)).sum()",
     "np.abs(np.diff(r)).sum()"),
]

_MODULE_RUNNER = """
import importlib.util, sys
sys.path.insert(0, {root!r})
import oracle
spec = importlib.util.spec_from_file_location("oracle.{name}", {path!r})
mod = importlib.util.module_from_spec(spec)
sys.modules["oracle.{name}"] = mod
spec.loader.exec_module(mod)
setattr(oracle, {name!r}, mod)
import pytest
sys.exit(pytest.main([*{tests!r}, "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"]))
"""


def _module_pins(folder, module, old, new, tests, env=None):
    """Run `tests` in a subprocess with oracle/<module>.py replaced by a copy with `old` -> `new`."""
    os.makedirs(folder)
    text = open(os.path.join(ORACLE, module + ".py")).read()
    if old is not None:
        assert text.count(old) == 1, f"{module}.py: the text to replace must occur once: {old!r}"
        text = text.replace(old, new)
    path = os.path.join(folder, module + ".py")
    open(path, "w").write(text)
    code = _MODULE_RUNNER.format(root=ROOT, name=module, path=path, tests=tests)
    res = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=600,
                         env=dict(os.environ, **(env or {})))
    return res.returncode, "\n".join((res.stdout + res.stderr).splitlines()[-15:])


def _riemann_pins(folder, old, new):
    return _module_pins(folder, "riemann", old, new, [os.path.join("tests", "test_riemann_cpu.py")])


@pytest.fixture(scope="module")
def riemann_outcomes(tmp_path_factory):
    base = tmp_path_factory.mktemp("riemann_mutants")
    cases = [("unmodified", None, None)] + RIEMANN_MUTANTS
    with ThreadPoolExecutor(max_workers=max(1, min(8, (os.cpu_count() or 2) // 2))) as pool:
        return dict(pool.map(lambda c: (c[0], _riemann_pins(str(base / c[0]), c[1], c[2])), cases))


def test_unmodified_riemann_checker_passes_its_pins(riemann_outcomes):
    status, tail = riemann_outcomes["unmodified"]
    assert status == 0, tail


@pytest.mark.parametrize("name", [m[0] for m in RIEMANN_MUTANTS])
def test_planted_mistake_in_the_riemann_checker_fails_a_pin(riemann_outcomes, name):
    status, tail = riemann_outcomes[name]
    assert status == 1, f"{name} was not caught by the Riemann pins (status {status}):\n{tail}"


# The oracle's Python face (oracle/oracle.py) is marshalling apart from one formula, the
# relaxation time of a viscosity (Sec. 1 with the 1/2 of Eq. 5's reading): planted in a copy
# loaded in place of the original, against the C library built from the unmodified sources.
def test_planted_mistake_in_the_viscosity_reading_fails_a_pin(tmp_path):
    from oracle import oracle as O

    lib = O.build()
    env = {"OLBM_ORACLE_LIB": lib, "OMP_NUM_THREADS": "2"}
    status, tail = _module_pins(str(tmp_path / "control"), "oracle", None, None, PINS, env=env)
    assert status == 0, tail  # the unmodified copy, loaded the same way, passes
    status, tail = _module_pins(str(tmp_path / "tau"), "oracle", "return nu / theta + 0.5", "return nu / theta",
                                PINS, env=env)
    assert status == 1, f"tau_from_nu without the 1/2 was not caught (status {status}):\n{tail}"
