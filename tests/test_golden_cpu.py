"""Checks against values the paper prints, transcribed under tests/golden/: the
numbering of the D2Q9 velocities in Fig. 1a (d2q9_velocities_fig1a.txt), which the
oracle must follow, and the set-ups of the Sec. 5 experiments
(sec5_experiment_setups.txt), which the experiment harness must run.

The oracle's C core holds its own velocity table. These tests read the figure's
numbering from the fixture and check that the oracle's populations follow it: the
guided equilibrium's moments taken with the figure's c_i are the ones Eqs. 3-4 fix,
and a population streams along the figure's c_i (Eq. 1b). A permuted or mirrored
table in the oracle fails them."""
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def fig1a():
    rows = []
    with open(os.path.join(HERE, "golden", "d2q9_velocities_fig1a.txt")) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append([int(v) for v in line.split()])
    table = np.array(rows, dtype=np.int64)
    assert table.shape == (9, 3) and (table[:, 0] == np.arange(9)).all()
    return table[:, 1], table[:, 2]


def test_fixture_is_the_d2q9_set():
    cx, cy = fig1a()
    assert sorted(zip(cx.tolist(), cy.tolist())) == sorted((a, b) for a in (-1, 0, 1) for b in (-1, 0, 1))


def test_oracle_velocity_table_is_fig1a(oracle):
    cx, cy = fig1a()
    np.testing.assert_array_equal(oracle.CX, cx)
    np.testing.assert_array_equal(oracle.CY, cy)


@pytest.mark.parametrize("rho,ux,uy,theta", [(1.0, 0.0, 0.0, 1 / 3), (1.3, 0.12, -0.07, 0.3),
                                             (0.8, -0.2, 0.15, 0.4), (1.1, 0.05, 0.3, 0.25)])
def test_equilibrium_moments_in_the_figure_numbering(oracle, rho, ux, uy, theta):
    """Eqs. 3-4: sum f = rho, sum c f = rho u, sum c_a c_b f = rho (theta delta_ab + u_a u_b),
    with c_i taken from the figure and f_i from the oracle's C core (Eq. 10)."""
    cx, cy = fig1a()
    f = np.asarray(oracle.geq(rho, ux, uy, theta), dtype=np.float64)
    tol = 1e-14
    assert abs(f.sum() - rho) < tol
    assert abs((cx * f).sum() - rho * ux) < tol and abs((cy * f).sum() - rho * uy) < tol
    assert abs((cx * cx * f).sum() - rho * (theta + ux * ux)) < tol
    assert abs((cy * cy * f).sum() - rho * (theta + uy * uy)) < tol
    assert abs((cx * cy * f).sum() - rho * ux * uy) < tol


@pytest.mark.parametrize("i", range(1, 9))
def test_population_streams_along_its_figure_velocity(oracle, i):
    """Eq. 1b: a bump in population i at node x0 of a fluid at rest is found at x0 + c_i
    one step later (tau large, so the collision barely touches the bump)."""
    cx, cy = fig1a()
    nx, ny, x0, y0, theta = 7, 6, 3, 2, 1 / 3
    f = np.array(oracle.init(np.ones((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx)), theta))
    base = f.copy()
    f[i, y0, x0] += 1e-3
    out = np.asarray(oracle.run(f, theta, 1e6, 0, 1))
    bump = np.abs(out[i] - base[i])
    y1, x1 = np.unravel_index(np.argmax(bump), bump.shape)
    assert (x1, y1) == ((x0 + cx[i]) % nx, (y0 + cy[i]) % ny)
    assert bump[y1, x1] > 0.9e-3


def sec5():
    out = {}
    with open(os.path.join(HERE, "golden", "sec5_experiment_setups.txt")) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                key, *vals = line.split()
                out[key] = [float(v) for v in vals]
    return out


def _defaults(fn):
    import inspect

    return {k: p.default for k, p in inspect.signature(fn).parameters.items() if p.default is not inspect._empty}


def test_experiment_set_ups_are_the_papers():
    """The experiment harness runs Sec. 5's set-ups: its defaults and case lists against the
    transcription of the values the paper prints."""
    pytest.importorskip("torch")
    from paper_2602_21242_gb300 import experiments as X

    g = sec5()
    sw = _defaults(X.rotated_shear_wave_viscosity)
    assert (sw["n"], sw["nu"], sw["a0"], sw["steps"]) == (g["shear_wave.N"][0], g["shear_wave.nu"][0],
                                                          g["shear_wave.A0"][0], g["shear_wave.iterations"][0])
    np.testing.assert_allclose(X.SHEAR_WAVE_THETAS, g["shear_wave.theta"], rtol=1e-15)
    rho, ux, uy = X.rotated_shear_wave_fields(int(g["shear_wave.N"][0]), 0.6, sw["a0"])
    assert (rho == g["shear_wave.rho"][0]).all()
    assert ux.mean() == pytest.approx(0.6 / np.sqrt(g["shear_wave.mean_flow_divisor_squared"][0]), rel=1e-14)
    st = _defaults(X.shocktube_run)
    assert (st["n"], st["steps"]) == (g["shocktube.nx"][0], g["shocktube.steps"][0])
    assert [list(c) for c in X.SHOCKTUBE_CASES] == [g["shocktube.case1"], g["shocktube.case2"]]
    sl = _defaults(X.shear_layer_run)
    assert (sl["kappa"], sl["delta"], sl["u0"], sl["re"], sl["turnovers"]) == (
        g["shear_layer.kappa"][0], g["shear_layer.delta"][0], g["shear_layer.u0"][0], g["shear_layer.Re"][0],
        g["shear_layer.turnovers"][0])
    assert list(X.SHEAR_LAYER_GRIDS) == g["shear_layer.N"] and list(X.SHEAR_LAYER_THETAS) == g["shear_layer.theta"]


def test_shear_layer_initial_condition():
    """Sec. 5.3's initial condition: u_x vanishes at y = N/4 and 3N/4, tends to +-u0 away from the
    layers and is mirrored about y = N/2; u_y = delta u0 sin(2 pi (x/N + 1/4)) peaks at x = 0."""
    pytest.importorskip("torch")
    from paper_2602_21242_gb300 import experiments as X

    g = sec5()
    n, u0, kappa, delta = 128, g["shear_layer.u0"][0], g["shear_layer.kappa"][0], g["shear_layer.delta"][0]
    rho, ux, uy = X.shear_layer_fields(n, u0, kappa, delta)
    assert (rho == 1.0).all() and rho.shape == (n, n)
    assert abs(ux[n // 4, 0]) < 1e-15 and abs(ux[3 * n // 4, 0]) < 1e-15
    assert ux[n // 2, 0] == pytest.approx(u0 * np.tanh(kappa / 4), rel=1e-14)
    assert ux[0, 0] == pytest.approx(-u0 * np.tanh(kappa / 4), rel=1e-14)
    np.testing.assert_allclose(ux[1:n // 2, 0], ux[n - 1:n // 2:-1, 0], rtol=0, atol=1e-17)
    assert (ux == ux[:, :1]).all() and (uy == uy[:1, :]).all()
    assert uy[0, 0] == pytest.approx(delta * u0, rel=1e-14) and abs(uy[0, n // 4]) < 1e-17
