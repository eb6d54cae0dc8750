"""The paper's benchmark experiments (arXiv 2602.21242, Sec. 5) run on the GPU path.

* Rotated decaying shear wave (Sec. 5.1, Fig. 2): numerical viscosity nu~/nu
  against Mach number for the four models and several temperatures. The paper
  runs a 1 x 200 grid (N = 200 nodes along y) with u_x = u_y = Ma/sqrt(6) +
  A0 sin[sqrt(2) pi (-x + y)/N]; with a single column this is a wave along y
  whose printed period (sqrt(2) N) does not fit the periodic N-node grid. Reading
  taken (orientation="axis", the default): nx = 1, ny = N, u_x = u_y = Ma/sqrt(6)
  + A0 sin(2 pi y / N) -- the mean flow points along the diagonal (the "pi/4
  rotation") and the transverse component u_x is a shear wave along y; nu~ is
  the decay rate of its Fourier coefficient divided by k^2 = (2 pi/N)^2. The
  alternative orientation="diagonal" runs an N x N grid with the wave along
  (-1, 1) and the perturbation along (1, 1) (k^2 = 2 (2 pi/N)^2), which also
  loads the normal-stress channel. Runs that become non-finite are reported as
  nu~ = 0 (the paper's convention for catastrophic instability); a growing
  amplitude gives a negative nu~.
* Isothermal shocktube (Sec. 5.2): an 800 x 1 grid closed by fullway
  bounce-back walls (x = 0 and x = 799 are wall nodes), a density jump in the
  middle of the fluid at rest, 400 steps, (theta, nu) = (0.4, 1e-12) and
  (0.55, 1e-9). The paper does not state the density ratio; reading taken:
  rho_L = 1.5, rho_R = 0.75 (ratio 2), jump between nodes 399 and 400. This
  module runs it and returns the fields; the tests compare them with the exact
  solution of the isothermal Euler Riemann problem (pressure p = theta rho,
  sound speed sqrt(theta)), which lives with the oracle.
* Doubly periodic shear layer (Sec. 5.3): the paper's initial condition
  (kappa = 80, delta = 0.05, u0 = 0.04, Re = u0 N / nu = 3e4) run to one turnover
  time N / u0; reports whether each model stays finite and the vorticity field.

All computation runs in liblbm.so; this module sets up inputs and reads moments.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .lattice import Lattice, tau_from_nu


def rotated_shear_wave_fields(n: int, ma: float, a0: float = 1e-3, orientation: str = "axis"):
    """(rho, u_x, u_y) of the rotated shear wave: (N, 1) arrays for "axis", (N, N) for "diagonal"."""
    if orientation == "axis":
        y = np.arange(n, dtype=np.float64)[:, None]
        u = ma / math.sqrt(6.0) + a0 * np.sin(2 * math.pi * y / n)
        return np.ones((n, 1)), u.copy(), u.copy()
    x = np.arange(n, dtype=np.float64)[None, :]
    y = np.arange(n, dtype=np.float64)[:, None]
    u = np.broadcast_to(ma / math.sqrt(6.0) + a0 * np.sin(2 * math.pi * (-x + y) / n), (n, n)).copy()
    return np.ones((n, n)), u, u.copy()


def shear_mode(ux, uy, n: int, orientation: str = "axis") -> complex:
    """Fourier coefficient of the shear wave: u_x on k = 2 pi / N along y ("axis"), or
    (u_x + u_y)/sqrt(2) on k = (2 pi / N)(-1, 1) ("diagonal")."""
    ux = ux.cpu().numpy() if isinstance(ux, torch.Tensor) else np.asarray(ux)
    uy = uy.cpu().numpy() if isinstance(uy, torch.Tensor) else np.asarray(uy)
    if orientation == "axis":
        return complex(np.fft.fft(ux[:, 0])[1])
    return complex(np.fft.fft2((ux + uy) / math.sqrt(2.0))[1, n - 1])  # index (k_y, k_x) = (1, -1)


def shear_k2(n: int, orientation: str = "axis") -> float:
    return (2 * math.pi / n) ** 2 * (1.0 if orientation == "axis" else 2.0)


def viscosity_from_amplitudes(a1: float, a2: float, dt: int, k2: float) -> float:
    """Viscosity of a shear wave whose mode amplitude fell from a1 to a2 over dt steps:
    |a(t)| = |a(0)| exp(-nu k^2 t), so nu = -ln(a2 / a1) / (dt k^2) (negative if it grew)."""
    return -math.log(a2 / a1) / (dt * k2)


def rotated_shear_wave_viscosity(model: str, theta: float, ma: float, n: int = 200, nu: float = 1e-3,
                                 steps: int = 1200, t_fit: int = 200, a0: float = 1e-3, prec: str = "f64",
                                 orientation: str = "axis", device=None):
    """Numerical viscosity ratio nu~/nu of the rotated shear wave (0.0 if the run became non-finite)."""
    tau = tau_from_nu(nu, theta)
    rho, ux, uy = rotated_shear_wave_fields(n, ma, a0, orientation)
    ny, nx = rho.shape
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else device
    with Lattice(nx, ny, theta, tau, model, prec, device=dev) as lat:
        lat.init(*(torch.from_numpy(a).to(dev) for a in (rho, ux, uy)))
        lat.step(t_fit)
        _, u1, v1 = lat.moments()
        a1 = abs(shear_mode(u1, v1, n, orientation))
        lat.step(steps - t_fit)
        r2, u2, v2 = lat.moments()
        if not (torch.isfinite(r2).all() and torch.isfinite(u2).all() and torch.isfinite(v2).all()):
            return 0.0
        a2 = abs(shear_mode(u2, v2, n, orientation))
    if not (a2 > 0 and a1 > 0):
        return 0.0
    return viscosity_from_amplitudes(a1, a2, steps - t_fit, shear_k2(n, orientation)) / nu


def shear_layer_fields(n: int, u0: float = 0.04, kappa: float = 80.0, delta: float = 0.05):
    """(rho, u_x, u_y) of the doubly periodic shear layer on an N x N grid (Sec. 5.3): unit density,
    u_x = u0 tanh(kappa (y/N - 1/4)) for y <= N/2 and u0 tanh(kappa (3/4 - y/N)) above, and
    u_y = delta u0 sin(2 pi (x/N + 1/4))."""
    y = np.arange(n, dtype=np.float64)[:, None]
    x = np.arange(n, dtype=np.float64)[None, :]
    ux = np.where(y <= n / 2, u0 * np.tanh(kappa * (y / n - 0.25)), u0 * np.tanh(kappa * (0.75 - y / n)))
    ux = np.broadcast_to(ux, (n, n)).copy()
    uy = np.broadcast_to(delta * u0 * np.sin(2 * math.pi * (x / n + 0.25)), (n, n)).copy()
    return np.ones((n, n)), ux, uy


def shear_layer_run(model: str, theta: float, n: int, u0: float = 0.04, kappa: float = 80.0, delta: float = 0.05,
                    re: float = 3.0e4, turnovers: float = 1.0, prec: str = "f64", device=None):
    """Paper's doubly periodic shear layer to `turnovers` x N/u0 steps. Returns (finite, steps,
    vorticity (ny, nx) float64 numpy array or None)."""
    nu = u0 * n / re
    tau = tau_from_nu(nu, theta)
    rho, ux, uy = shear_layer_fields(n, u0, kappa, delta)
    steps = int(round(turnovers * n / u0))
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else device
    with Lattice(n, n, theta, tau, model, prec, device=dev) as lat:
        lat.init(*(torch.from_numpy(a).to(dev) for a in (rho, ux, uy)))
        lat.step(steps)
        r, u, v = (t.cpu().numpy() for t in lat.moments())
    finite = bool(np.isfinite(r).all() and np.isfinite(u).all() and np.isfinite(v).all())
    if not finite:
        return False, steps, None
    # vorticity by periodic central differences (lattice units)
    w = (np.roll(v, -1, axis=1) - np.roll(v, 1, axis=1)) / 2 - (np.roll(u, -1, axis=0) - np.roll(u, 1, axis=0)) / 2
    return True, steps, w


SHOCKTUBE_RHO = (1.5, 0.75)

# The runs of Sec. 5 as the paper sets them up: the temperatures of the rotated shear wave
# (Sec. 5.1, Fig. 2), the (theta, nu) pairs of the shocktube (Sec. 5.2) and the grids and
# temperatures of the shear layer (Sec. 5.3).
SHEAR_WAVE_THETAS = (0.25, 1.0 / 3.0, 0.4, 0.5)
SHOCKTUBE_CASES = ((0.4, 1e-12), (0.55, 1e-9))
SHEAR_LAYER_GRIDS = (128, 256, 512)
SHEAR_LAYER_THETAS = (0.4, 0.6)


def shocktube_fields(n: int = 800, rho_l: float = SHOCKTUBE_RHO[0], rho_r: float = SHOCKTUBE_RHO[1]):
    """(rho, u_x, u_y) as (1, n) arrays and the (1, n) wall mask: wall nodes 0 and n - 1, rho_l on
    nodes 1 .. n/2 - 1, rho_r on n/2 .. n - 2, fluid at rest (wall nodes carry rho_l / rho_r at rest)."""
    x = np.arange(n)
    rho = np.where(x < n // 2, rho_l, rho_r).astype(np.float64)[None, :]
    walls = np.zeros((1, n), dtype=np.uint8)
    walls[0, 0] = walls[0, n - 1] = 1
    return rho, np.zeros((1, n)), np.zeros((1, n)), walls


def shocktube_run(model: str, theta: float, nu: float, n: int = 800, steps: int = 400,
                  rho_l: float = SHOCKTUBE_RHO[0], rho_r: float = SHOCKTUBE_RHO[1], prec: str = "f64",
                  device=None):
    """Paper's isothermal shocktube on the GPU path. Returns a dict with the fluid nodes' x, rho and
    u_x after `steps` steps, whether they stayed finite, the position x0 of the initial jump (between
    nodes n/2 - 1 and n/2) and the set-up (theta, steps, rho_l, rho_r) that a comparison with the
    exact solution needs."""
    tau = tau_from_nu(nu, theta)
    rho0, ux0, uy0, walls = shocktube_fields(n, rho_l, rho_r)
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else device
    with Lattice(n, 1, theta, tau, model, prec, device=dev) as lat:
        lat.set_walls(walls)
        lat.init(*(torch.from_numpy(a).to(dev) for a in (rho0, ux0, uy0)))
        lat.step(steps)
        r, u, _ = (t.cpu().numpy()[0] for t in lat.moments())
    fluid = np.arange(1, n - 1)
    r, u = r[fluid], u[fluid]
    return {"x": fluid, "rho": r, "ux": u, "finite": bool(np.isfinite(r).all() and np.isfinite(u).all()),
            "x0": n // 2 - 0.5, "theta": theta, "steps": steps, "rho_l": rho_l, "rho_r": rho_r}


__all__ = ["rotated_shear_wave_fields", "rotated_shear_wave_viscosity", "shear_mode", "shear_k2",
           "viscosity_from_amplitudes", "shear_layer_fields", "shear_layer_run", "shocktube_fields", "shocktube_run",
           "SHOCKTUBE_RHO", "SHEAR_WAVE_THETAS", "SHOCKTUBE_CASES", "SHEAR_LAYER_GRIDS", "SHEAR_LAYER_THETAS"]
