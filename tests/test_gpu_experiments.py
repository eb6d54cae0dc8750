"""The paper's benchmark experiments on the GPU path (Sec. 5): the measured
quantities agree with the same measurement made on the oracle, and the
qualitative outcomes the paper reports hold where this build reproduces them."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import riemann
from paper_2602_21242_gb300 import experiments
from paper_2602_21242_gb300.lattice import tau_from_nu

pytestmark = pytest.mark.gpu


def oracle_nu_ratio(oracle, model, theta, ma, n, nu, steps, t_fit, orientation):
    m = {"lbgk": 0, "oreg": 1, "partial": 2, "complete": 3, "complete_neq": 4, "lbgk_poly": 5}[model]
    tau = tau_from_nu(nu, theta)
    rho, ux, uy = experiments.rotated_shear_wave_fields(n, ma, orientation=orientation)
    f = oracle.run(oracle.init(rho, ux, uy, theta), theta, tau, m, t_fit)
    _, u1, v1 = oracle.moments(f)
    f = oracle.run(f, theta, tau, m, steps - t_fit)
    _, u2, v2 = oracle.moments(f)
    a1 = abs(experiments.shear_mode(u1, v1, n, orientation))
    a2 = abs(experiments.shear_mode(u2, v2, n, orientation))
    return -math.log(a2 / a1) / ((steps - t_fit) * experiments.shear_k2(n, orientation)) / nu


@pytest.mark.parametrize("orientation", ["axis", "diagonal"])
@pytest.mark.parametrize("model", ["lbgk", "oreg", "partial", "complete", "complete_neq", "lbgk_poly"])
def test_rotated_shear_wave_measurement_matches_oracle(oracle, model, orientation):
    n, theta, ma, nu, steps, t_fit = 32, 0.4, 0.3, 0.005, 300, 50
    got = experiments.rotated_shear_wave_viscosity(model, theta, ma, n=n, nu=nu, steps=steps, t_fit=t_fit,
                                                   orientation=orientation)
    want = oracle_nu_ratio(oracle, model, theta, ma, n, nu, steps, t_fit, orientation)
    assert got == pytest.approx(want, rel=1e-8)


def test_corrected_models_recover_the_viscosity():
    """Sec. 5.1: the partially and completely corrected models recover nu over the Mach range
    (paper: up to Ma = 1, 0.9, 0.4 at theta = 1/3, 0.4, 0.5), the complete one also at
    theta = 0.25 over the whole range."""
    cases = [(1.0 / 3.0, (0.1, 0.5, 0.9), ("partial", "complete")), (0.4, (0.1, 0.5, 0.9), ("partial", "complete")),
             (0.5, (0.1, 0.4), ("partial", "complete")), (0.25, (0.1, 0.5, 0.9), ("complete",))]
    for theta, mas, models in cases:
        for model in models:
            for ma in mas:
                r = experiments.rotated_shear_wave_viscosity(model, theta, ma)
                assert r == pytest.approx(1.0, abs=0.03), (model, theta, ma, r)


def test_lbgk_readings_and_orientations():
    """Sec. 5.1's statements on LBGK under the readings this build can take (recorded, not the
    paper's data): on the column (wave along y) LBGK on the GEq recovers nu at theta = 0.25, while
    with the wave along the lattice diagonal, which loads the normal-stress channel, it stays
    stable at every Ma but misses nu (the paper: stable, viscosity wrong at all Ma); the polynomial
    equilibrium (LBM_LBGK_POLY) on the column gives nu~ falling with Ma at theta = 1/3."""
    axis = [experiments.rotated_shear_wave_viscosity("lbgk", 0.25, ma) for ma in (0.1, 0.5, 1.0)]
    assert all(abs(r - 1.0) < 0.01 for r in axis), axis
    diag = [experiments.rotated_shear_wave_viscosity("lbgk", 0.25, ma, orientation="diagonal") for ma in (0.1, 1.0)]
    assert all(r > 0 and abs(r - 1.0) > 0.3 for r in diag), diag
    poly = [experiments.rotated_shear_wave_viscosity("lbgk_poly", 1.0 / 3.0, ma) for ma in (0.1, 0.4, 0.7)]
    assert abs(poly[0] - 1.0) < 0.02 and poly[0] > poly[1] > poly[2] > 0, poly


def test_uncorrected_model_degrades_with_mach_and_temperature():
    """Sec. 5.1: the uncorrected model recovers nu only at small Ma, over a range that shrinks as
    theta grows, and is not stable at theta = 0.25."""
    assert experiments.rotated_shear_wave_viscosity("oreg", 1.0 / 3.0, 0.1) == pytest.approx(1.0, abs=0.03)
    assert abs(experiments.rotated_shear_wave_viscosity("oreg", 1.0 / 3.0, 0.7) - 1.0) > 0.5
    assert abs(experiments.rotated_shear_wave_viscosity("oreg", 0.4, 0.5) - 1.0) > 0.5
    assert experiments.rotated_shear_wave_viscosity("oreg", 0.25, 0.1) == 0.0


def test_shear_layer_lbgk_fails_where_oreg_holds():
    """Sec. 5.3: at theta = 0.6 LBGK does not give a physical shear layer on N = 128 while the
    corrected OReg model stays bounded."""
    ok_l, _, w_l = experiments.shear_layer_run("lbgk", 0.6, 128)
    ok_c, _, w_c = experiments.shear_layer_run("complete", 0.6, 128)
    assert ok_c and np.abs(w_c).max() < 0.05
    assert (not ok_l) or np.abs(w_l).max() > 1.0


def test_shocktube_matches_the_paper_statements():
    """Sec. 5.2, (theta, nu) = (0.4, 1e-12): LBGK shows large oscillations; the uncorrected model is
    free of them but its middle-state density is low while its velocity is right; the partially and
    completely corrected models recover the exact middle state. (0.55, 1e-9): LBGK is unphysical; the
    uncorrected model keeps its deficiency; the corrected ones stay accurate, oscillations small."""
    r = {m: riemann.shocktube_measures(experiments.shocktube_run(m, 0.4, 1e-12))
         for m in ("lbgk", "oreg", "partial", "complete")}
    rs, us = r["oreg"]["rho_star"], r["oreg"]["u_star"]
    assert r["lbgk"]["tv_excess"] > 1.0
    assert r["oreg"]["tv_excess"] < 0.02
    assert rs - r["oreg"]["plateau_rho"] > 2e-3 and abs(r["oreg"]["plateau_ux"] - us) < 1e-3
    for m in ("partial", "complete"):
        assert abs(r[m]["plateau_rho"] - rs) < 2e-4 and abs(r[m]["plateau_ux"] - us) < 2e-4
        assert r[m]["tv_excess"] < 0.02 and r[m]["l1_rho"] < 0.5 * r["oreg"]["l1_rho"]
    r = {m: riemann.shocktube_measures(experiments.shocktube_run(m, 0.55, 1e-9))
         for m in ("lbgk", "oreg", "partial", "complete")}
    assert (not r["lbgk"]["finite"]) or r["lbgk"]["l1_rho"] > 1.0
    assert rs - r["oreg"]["plateau_rho"] > 2e-3
    for m in ("partial", "complete"):
        assert abs(r[m]["plateau_rho"] - rs) < 2e-4 and r[m]["tv_excess"] < 0.2
