"""Host-side parts of the rotated decaying shear wave (Sec. 5.1) that need no GPU: the
initial fields, the Fourier mode whose decay gives nu~, its wavenumber and the decay
formula, checked against closed forms of a single sine mode."""
import math

import numpy as np
import pytest

pytest.importorskip("torch")

from paper_2602_21242_gb300 import experiments as X  # noqa: E402


@pytest.mark.parametrize("orientation", ["axis", "diagonal"])
def test_initial_fields(orientation):
    """Mean flow u_x = u_y = Ma/sqrt(6) along the diagonal plus the A0 sine; rho = 1."""
    n, ma, a0 = 40, 0.3, 1e-3
    rho, ux, uy = X.rotated_shear_wave_fields(n, ma, a0, orientation)
    assert rho.shape == ux.shape == uy.shape == ((n, 1) if orientation == "axis" else (n, n))
    assert (rho == 1.0).all()
    np.testing.assert_allclose(ux.mean(), ma / math.sqrt(6.0), rtol=1e-14)
    np.testing.assert_allclose(ux - ma / math.sqrt(6.0), uy - ma / math.sqrt(6.0), atol=0)
    assert np.abs(ux - ma / math.sqrt(6.0)).max() == pytest.approx(a0, rel=1e-3)


def test_axis_mode_is_the_sine_amplitude():
    """u_x = A0 sin(2 pi y / N) has the Fourier coefficient -i A0 N / 2 at k = 2 pi / N; the
    mean flow sits at k = 0 and does not leak into it."""
    n, a0 = 64, 2e-3
    _, ux, uy = X.rotated_shear_wave_fields(n, 0.5, a0, "axis")
    c = X.shear_mode(ux, uy, n, "axis")
    assert c.real == pytest.approx(0.0, abs=1e-12) and c.imag == pytest.approx(-a0 * n / 2, rel=1e-12)
    assert X.shear_k2(n, "axis") == pytest.approx((2 * math.pi / n) ** 2, rel=1e-15)


def test_diagonal_mode_is_the_sine_amplitude():
    """(u_x + u_y)/sqrt(2) = sqrt(2) A0 sin(2 pi (-x + y)/N) + const has the coefficient
    -i sqrt(2) A0 N^2 / 2 at (k_y, k_x) = (1, -1), and |k|^2 = 2 (2 pi / N)^2."""
    n, a0 = 32, 1e-3
    _, ux, uy = X.rotated_shear_wave_fields(n, 0.7, a0, "diagonal")
    c = X.shear_mode(ux, uy, n, "diagonal")
    assert abs(c) == pytest.approx(math.sqrt(2) * a0 * n * n / 2, rel=1e-12)
    assert c.imag == pytest.approx(-math.sqrt(2) * a0 * n * n / 2, rel=1e-12)
    assert X.shear_k2(n, "diagonal") == pytest.approx(2 * (2 * math.pi / n) ** 2, rel=1e-15)


@pytest.mark.parametrize("orientation", ["axis", "diagonal"])
def test_decay_formula_recovers_a_known_viscosity(orientation):
    """A mode damped by exp(-nu k^2 t) over dt steps gives back nu; a growing one a negative nu."""
    n, a0, nu, dt = 50, 1e-3, 3.7e-3, 1000
    k2 = X.shear_k2(n, orientation)
    _, ux, uy = X.rotated_shear_wave_fields(n, 0.2, a0, orientation)
    mean = 0.2 / math.sqrt(6.0)
    damp = math.exp(-nu * k2 * dt)
    a1 = abs(X.shear_mode(ux, uy, n, orientation))
    a2 = abs(X.shear_mode(mean + (ux - mean) * damp, mean + (uy - mean) * damp, n, orientation))
    assert X.viscosity_from_amplitudes(a1, a2, dt, k2) == pytest.approx(nu, rel=1e-9)
    assert X.viscosity_from_amplitudes(a2, a1, dt, k2) == pytest.approx(-nu, rel=1e-9)


@pytest.mark.parametrize("orientation", ["axis", "diagonal"])
def test_viscosity_measurement_with_a_stand_in_lattice(monkeypatch, orientation):
    """The measurement's plumbing (init, steps to t_fit and on, moments, mode amplitudes, fit)
    on a stand-in lattice whose shear wave decays exactly at the lattice viscosity
    theta (tau - 1/2): the ratio comes out 1, and 0 once the fields turn non-finite."""
    import torch

    class Decaying:
        blow_up = False

        def __init__(self, nx, ny, theta, tau, model, prec, device=None):
            self.nu, self.t = theta * (tau - 0.5), 0
            self.k2 = X.shear_k2(ny, orientation)

        def __enter__(self):
            return self

        def __exit__(self, *exc):
            return False

        def init(self, rho, ux, uy):
            self.rho, self.ux, self.uy = rho.clone(), ux.clone(), uy.clone()
            self.mean = float(ux.mean())

        def step(self, n):
            self.t += n

        def moments(self):
            damp = math.exp(-self.nu * self.k2 * self.t)
            ux = self.mean + (self.ux - self.mean) * damp
            uy = self.mean + (self.uy - self.mean) * damp
            if Decaying.blow_up and self.t > 200:
                ux = ux * float("nan")
            return self.rho, ux, uy

    monkeypatch.setattr(X, "Lattice", Decaying)
    cpu = torch.device("cpu")
    ratio = X.rotated_shear_wave_viscosity("complete", 0.4, 0.5, n=40, nu=2e-3, orientation=orientation, device=cpu)
    assert ratio == pytest.approx(1.0, rel=1e-9)
    Decaying.blow_up = True
    assert X.rotated_shear_wave_viscosity("complete", 0.4, 0.5, n=40, nu=2e-3, orientation=orientation,
                                          device=cpu) == 0.0


def test_shear_layer_run_with_a_stand_in_lattice(monkeypatch):
    """The shear layer's plumbing (fields, viscosity from Re, one turnover of steps, vorticity) on
    a stand-in lattice that keeps its initial fields: the vorticity is that of the initial shear."""
    import torch

    seen = {}

    class Frozen:
        def __init__(self, nx, ny, theta, tau, model, prec, device=None):
            seen["tau"], seen["steps"] = tau, 0

        def __enter__(self):
            return self

        def __exit__(self, *exc):
            return False

        def init(self, rho, ux, uy):
            self.fields = (rho, ux, uy)

        def step(self, n):
            seen["steps"] += n

        def moments(self):
            return self.fields

    monkeypatch.setattr(X, "Lattice", Frozen)
    n, theta = 64, 0.4
    finite, steps, w = X.shear_layer_run("complete", theta, n, device=torch.device("cpu"))
    assert finite and steps == seen["steps"] == round(n / 0.04)
    assert seen["tau"] == pytest.approx(0.04 * n / 3.0e4 / theta + 0.5, rel=1e-15)
    _, ux, uy = X.shear_layer_fields(n)
    dudy = (np.roll(ux, -1, axis=0) - np.roll(ux, 1, axis=0)) / 2
    dvdx = (np.roll(uy, -1, axis=1) - np.roll(uy, 1, axis=1)) / 2
    np.testing.assert_allclose(w, dvdx - dudy, rtol=0, atol=1e-18)


def test_shocktube_run_with_a_stand_in_lattice(monkeypatch):
    """The shocktube's plumbing (walls at both ends, the density jump, the fluid nodes returned
    with the jump position and the set-up) on a stand-in lattice that keeps its initial fields."""
    import torch

    seen = {}

    class Frozen:
        def __init__(self, nx, ny, theta, tau, model, prec, device=None):
            seen["shape"], seen["tau"] = (ny, nx), tau

        def __enter__(self):
            return self

        def __exit__(self, *exc):
            return False

        def set_walls(self, mask):
            seen["walls"] = np.flatnonzero(mask)

        def init(self, rho, ux, uy):
            self.fields = (rho, ux, uy)

        def step(self, n):
            seen["steps"] = n

        def moments(self):
            return self.fields

    monkeypatch.setattr(X, "Lattice", Frozen)
    r = X.shocktube_run("complete", 0.4, 1e-12, device=torch.device("cpu"))
    assert seen["shape"] == (1, 800) and list(seen["walls"]) == [0, 799] and seen["steps"] == 400
    assert seen["tau"] == pytest.approx(1e-12 / 0.4 + 0.5, rel=1e-15)
    assert r["finite"] and list(r["x"]) == list(range(1, 799)) and r["x0"] == pytest.approx(399.5)
    assert (r["rho"][r["x"] < 400] == 1.5).all() and (r["rho"][r["x"] >= 400] == 0.75).all()
    assert (r["theta"], r["steps"], r["rho_l"], r["rho_r"]) == (0.4, 400, 1.5, 0.75)
