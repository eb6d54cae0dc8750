"""The exact isothermal Riemann solution that the shocktube experiment (Sec. 5.2) is measured
against, pinned to the Euler equations it solves: Rankine-Hugoniot jump conditions, the
rarefaction's Riemann invariant, closed forms of the symmetric problems, and conservation of
the integrals of rho and rho u over the whole wave pattern."""
import math

import numpy as np
import pytest

from oracle import riemann as ex


@pytest.mark.parametrize("theta", [0.4, 0.55, 1.0 / 3.0])
@pytest.mark.parametrize("rho_l,rho_r", [(1.5, 0.75), (1.0, 0.125), (0.6, 2.4)])
def test_shock_satisfies_rankine_hugoniot(theta, rho_l, rho_r):
    """Across the shock (speed s): s [rho] = [rho u] and s [rho u] = [rho u^2 + theta rho]."""
    rs, us = ex.isothermal_riemann(rho_l, rho_r, theta)
    c = math.sqrt(theta)
    if rho_l > rho_r:  # right-going shock into the right state
        s, (ra, ua), (rb, ub) = c * math.sqrt(rs / rho_r), (rs, us), (rho_r, 0.0)
    else:  # left-going shock into the left state
        s, (ra, ua), (rb, ub) = -c * math.sqrt(rs / rho_l), (rho_l, 0.0), (rs, us)
    assert s * (rb - ra) == pytest.approx(rb * ub - ra * ua, abs=1e-14)
    assert s * (rb * ub - ra * ua) == pytest.approx(rb * ub * ub + theta * rb - ra * ua * ua - theta * ra, abs=1e-14)


@pytest.mark.parametrize("theta", [0.4, 0.55])
def test_rarefaction_invariant_and_characteristics(theta):
    """Inside the left rarefaction u - c = xi and u + c ln rho equals its left-state value."""
    rho_l, rho_r, c = 1.5, 0.75, math.sqrt(theta)
    rs, us = ex.isothermal_riemann(rho_l, rho_r, theta)
    xi = np.linspace(-c + 1e-6, us - c - 1e-6, 50)
    rho, u = ex.isothermal_riemann_sample(rho_l, rho_r, theta, xi)
    np.testing.assert_allclose(u - c, xi, rtol=0, atol=1e-15)
    np.testing.assert_allclose(u + c * np.log(rho), c * math.log(rho_l), rtol=1e-14)
    # continuous at both edges of the fan
    assert ex.isothermal_riemann_sample(rho_l, rho_r, theta, [us - c])[0][0] == pytest.approx(rs, rel=1e-12)


@pytest.mark.parametrize("theta", [0.4, 0.55])
def test_right_rarefaction_invariant_and_characteristics(theta):
    """Mirror of the left fan (rho_l < rho_r): inside the right rarefaction u + c = xi and
    u - c ln rho equals its right-state value."""
    rho_l, rho_r, c = 0.6, 2.4, math.sqrt(theta)
    rs, us = ex.isothermal_riemann(rho_l, rho_r, theta)
    xi = np.linspace(us + c + 1e-6, c - 1e-6, 50)
    rho, u = ex.isothermal_riemann_sample(rho_l, rho_r, theta, xi)
    np.testing.assert_allclose(u + c, xi, rtol=0, atol=1e-15)
    np.testing.assert_allclose(u - c * np.log(rho), -c * math.log(rho_r), rtol=1e-14)
    assert ex.isothermal_riemann_sample(rho_l, rho_r, theta, [us + c])[0][0] == pytest.approx(rs, rel=1e-12)


def test_symmetric_problems_have_closed_forms():
    """Equal densities: colliding streams (u_l = -u_r = U) give two shocks with u* = 0 and
    sqrt(rho*/rho) = (U/c + sqrt((U/c)^2 + 4))/2; receding streams give two rarefactions with
    rho* = rho exp(-U/c); equal states at rest give rho* = rho, u* = 0."""
    theta, rho, U = 0.4, 1.2, 0.3
    c = math.sqrt(theta)
    rs, us = ex.isothermal_riemann(rho, rho, theta, U, -U)
    s = (U / c + math.sqrt((U / c) ** 2 + 4)) / 2
    assert rs == pytest.approx(rho * s * s, rel=1e-14) and us == pytest.approx(0.0, abs=1e-15)
    rs, us = ex.isothermal_riemann(rho, rho, theta, -U, U)
    assert rs == pytest.approx(rho * math.exp(-U / c), rel=1e-14) and us == pytest.approx(0.0, abs=1e-15)
    assert ex.isothermal_riemann(rho, rho, theta) == pytest.approx((rho, 0.0), abs=1e-15)


@pytest.mark.parametrize("theta", [0.4, 0.55])
@pytest.mark.parametrize("rho_l,rho_r", [(1.5, 0.75), (0.6, 2.4)])
def test_integrals_of_mass_and_momentum(theta, rho_l, rho_r):
    """On a domain wider than the wave pattern: the integral of rho stays at its initial value and the
    integral of rho u grows at the pressure difference, theta (rho_l - rho_r) per unit time. Both
    orientations: a left rarefaction with a right shock, and a left shock with a right rarefaction."""
    t = 1.0
    x = np.linspace(-2.0, 2.0, 400001)
    rho, u = ex.isothermal_riemann_sample(rho_l, rho_r, theta, x / t)
    h = x[1] - x[0]
    mass0 = 2.0 * rho_l + 2.0 * rho_r
    trapezoid = getattr(np, "trapezoid", None) or np.trapz
    assert trapezoid(rho, dx=h) == pytest.approx(mass0, rel=2e-6)
    assert trapezoid(rho * u, dx=h) == pytest.approx(theta * (rho_l - rho_r) * t, rel=2e-5)


def test_measures_of_the_exact_profile():
    """shocktube_measures on a run that equals the exact solution at its nodes: no l1 error, no
    total-variation excess, and the plateau at the middle state."""
    theta, steps, n = 0.4, 400, 800
    x = np.arange(1, n - 1)
    x0 = n // 2 - 0.5
    rho, u = ex.isothermal_riemann_sample(1.5, 0.75, theta, (x - x0) / steps)
    m = ex.shocktube_measures({"x": x, "rho": rho, "ux": u, "finite": True, "x0": x0, "theta": theta,
                               "steps": steps, "rho_l": 1.5, "rho_r": 0.75})
    assert m["l1_rho"] == 0.0 and m["l1_ux"] == 0.0 and abs(m["tv_excess"]) < 1e-12
    assert m["plateau_rho"] == pytest.approx(m["rho_star"], rel=1e-14)
    assert m["plateau_ux"] == pytest.approx(m["u_star"], rel=1e-14)
    bad = ex.shocktube_measures({"x": x, "rho": rho, "ux": u, "finite": False, "x0": x0, "theta": theta,
                                 "steps": steps, "rho_l": 1.5, "rho_r": 0.75})
    assert not bad["finite"] and "l1_rho" not in bad
    # a run off the exact profile by +-d at alternate nodes: l1 error exactly d, and the
    # oscillation shows up as total variation above the exact profile's: each step of the run
    # is at least 2 d - |exact step|, so the excess is at least 2 d (n - 1) - 2 TV(exact)
    d = 0.01
    sign = np.where(x % 2 == 0, 1.0, -1.0)
    off = ex.shocktube_measures({"x": x, "rho": rho + d * sign, "ux": u - d * sign, "finite": True, "x0": x0,
                                 "theta": theta, "steps": steps, "rho_l": 1.5, "rho_r": 0.75})
    assert off["l1_rho"] == pytest.approx(d, rel=1e-9) and off["l1_ux"] == pytest.approx(d, rel=1e-9)
    assert off["tv_excess"] >= 2 * d * (len(x) - 1) - 2 * np.abs(np.diff(rho)).sum() - 1e-9


def test_shocktube_fields_layout():
    pytest.importorskip("torch")
    from paper_2602_21242_gb300 import experiments

    rho, ux, uy, walls = experiments.shocktube_fields(800)
    assert rho.shape == ux.shape == uy.shape == walls.shape == (1, 800)
    assert walls[0, 0] == 1 and walls[0, 799] == 1 and walls.sum() == 2
    assert (rho[0, :400] == 1.5).all() and (rho[0, 400:] == 0.75).all()
