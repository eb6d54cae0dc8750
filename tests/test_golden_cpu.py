"""The oracle against the one table of values the paper prints: the numbering of the
D2Q9 velocities in Fig. 1a (tests/golden/d2q9_velocities_fig1a.txt).

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
